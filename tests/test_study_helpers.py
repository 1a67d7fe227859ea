"""Host-side helpers of the study drivers (no GPU): vorticity and vortex-blob counting of the
shear-layer study, the channel perturbation shapes, and the shear-layer input."""
import math

import numpy as np

import workloads as W
from paper_2410_09739_gb300 import channel_les_study as CH
from paper_2410_09739_gb300 import shear_layer_study as SL


def test_vorticity_of_solid_body_rotation():
    L, U = 64, 0.1
    c = np.arange(L) - L / 2 + 0.5
    x, y = np.meshgrid(c, c)
    w = 1e-3
    ux, uy = -w * y, w * x
    om = SL.vorticity(ux, uy, L, U)
    inner = om[2:-2, 2:-2]  # away from the periodic seam
    assert np.allclose(inner, 2 * w * L / U)


def test_blobs_are_periodic_connected_regions():
    m = np.zeros((8, 8), bool)
    m[0, 0] = m[0, 7] = m[7, 0] = True  # one region across both seams
    m[4, 4] = m[4, 5] = True           # a second one
    m[2, 2] = True                     # a third; diagonal neighbours do not connect
    m[3, 3] = True
    assert SL.blobs(m) == 4


def test_shear_layer_input_rolls_up_into_one_blob_per_sign():
    ux, uy = W.shear_layers(128, 0.1)[1:]
    om = SL.vorticity(ux, uy, 128, 0.1)
    assert SL.cores(SL.sample64(om, 128)) == [1, 1]
    # the two layers carry opposite vorticity
    assert np.max(om) > 0 > np.min(om)


def test_half_channel_perturbation_respects_wall_and_symmetry_plane():
    nx, ny, nz, H = 16, 32, 12, 32
    du, dv, dw = CH.perturbation(nx, ny, nz, H, 1.0)
    y = (np.arange(ny) + 0.5) / H
    # amplitudes of the wall-normal shapes at the first and last rows
    assert np.max(np.abs(du[:, 0, :])) < 0.06 and np.max(np.abs(dv[:, 0, :])) < 0.06
    assert np.max(np.abs(dv[:, -1, :])) < 0.06  # v' vanishes at the symmetry plane
    assert np.max(np.abs(du[:, -1, :])) > 0.95  # u' is largest there
    assert np.allclose(np.max(np.abs(du), axis=(0, 2)), np.sin(0.5 * math.pi * y), atol=1e-2)


def test_full_channel_perturbation_crosses_the_centre_plane():
    nx, ny, nz = 16, 32, 12
    du, dv, dw = CH.perturbation(nx, ny, nz, ny, 1.0, full=True)
    assert np.max(np.abs(dv[:, ny // 2, :])) > 0.3  # v' does not vanish at the centre
    assert np.max(np.abs(du[:, 0, :])) < 0.06 and np.max(np.abs(du[:, -1, :])) < 0.06


def test_cavity2d_vortex_centres_of_a_synthetic_stream_function():
    from paper_2410_09739_gb300 import cavity2d_study as C2
    L = 200
    c = (np.arange(L) + 0.5) / L
    x, y = np.meshgrid(c, c)

    def well(x0, y0, a, s):
        return a * np.exp(-((x - x0) ** 2 + (y - y0) ** 2) / s ** 2)

    psi = well(0.531, 0.565, -0.1, 0.2) + well(0.864, 0.112, 1e-3, 0.03) + well(0.083, 0.077, 1e-4, 0.02)
    cen = C2.vortex_centres(psi)
    assert abs(cen["PV"][0] - 0.531) < 2e-3 and abs(cen["PV"][1] - 0.565) < 2e-3
    assert abs(cen["BR1"][0] - 0.864) < 3e-3 and abs(cen["BR1"][1] - 0.112) < 3e-3
    assert abs(cen["BL"][0] - 0.083) < 3e-3 and abs(cen["BL"][1] - 0.077) < 3e-3


def test_cavity2d_stream_function_integrates_u():
    from paper_2410_09739_gb300 import cavity2d_study as C2
    ux = np.ones((10, 3))
    psi = C2.stream_function(ux)
    assert np.allclose(psi[:, 0], np.arange(10) + 0.5)
