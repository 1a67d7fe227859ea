"""What the trained closure network gains over the method without it.

Decaying turbulence, the case an eddy-viscosity closure is made for: the Taylor-Green vortex at
Re = 1600 on a periodic 256^3 grid, box-filtered onto 128^3 (r = 2, acoustic scaling, the same Re
on both grids) every half convective time for 15 convective times.  The network is trained on
those snapshots by the library's own tensor-core training kernels; three coarse runs start from
the filtered initial field: plain FPC-LBM, FPC-LBM with the learned correction, and FPC-LBM with
the Smagorinsky model (C_s = 0.1, no walls).  Past the transition the plain coarse run keeps too
much kinetic energy (it lacks the sub-filter dissipation); the learned correction supplies it.

Measured on one GB300 (both training seeds tried): RMS over the snapshots of
KE_coarse / KE_filtered - 1 = 0.0655 plain, 0.0531 learned, 0.0531 Smagorinsky; the network
explains 40 % of the label variance (standardised training loss 0.60).  The test asks for a gain of
at least 10 % over plain and for the learned run to stay within 15 % of the Smagorinsky run, the
paper's own subgrid model (Sec. 4).  Everything in the pipeline is deterministic (fixed-order
reductions, no atomics in training), so the numbers repeat from run to run.

(At r = 4 the coarse grid's own numerical dissipation already exceeds the sub-filter dissipation
before the transition, so both closures make the energy history worse there; this is measured
and reported with the studies.)
"""
import pytest

pytestmark = pytest.mark.gpu


def test_learned_closure_gain_in_decaying_turbulence():
    pytest.importorskip("torch")
    from paper_2410_09739_gb300 import closure_study as CS
    out = CS.decay(CS.parse(["--flow", "tgv", "--fine", "256", "256", "256", "--r", "2", "--re", "1600",
                             "--t-end", "15", "--dt", "0.5", "--precision", "fp32", "--epochs", "20",
                             "--seed", "1"]))
    runs = out["coarse"]
    assert all(r["status"] == "ok" for r in runs.values()), {k: r["status"] for k, r in runs.items()}
    e = out["errors"]
    print("KE rel. RMS error: plain %.4f learned %.4f smagorinsky %.4f" % (e["plain"], e["learned"],
                                                                         e["smagorinsky"]))
    # training loss on the standardised label (a constant predictor scores 1): measured 0.60
    assert out["training"]["loss_last"] < 0.8
    assert e["learned"] <= 0.9 * e["plain"]
    assert e["learned"] <= 1.15 * e["smagorinsky"]
