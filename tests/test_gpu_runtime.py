"""Host runtime: bit-identical checkpoint and resume through the raw state, allocation failures
injected on the host, and guard bands around the populations.

* Resume: a run of 2n steps and a run of n steps, checkpointed with fpclbm_get_state, restored
  into a fresh handle with fpclbm_set_state and continued for n steps, end in the same stored
  bytes, in every storage type and at both AA parities (odd and even n), including the
  captured-graph path (n >= 32).
* Allocation failures: the library's allocation wrapper is told to fail the k-th next allocation
  (fpclbm_test_alloc_hook); every create path and the closure's training scratch must then return
  FPCLBM_ERR_ALLOC, leave the count of live allocations where it was, and leave the library
  usable.  Nothing fails on the GPU: the failure is made on the host, before the CUDA call.
* Guard bands: every slot row is padded to a multiple of 64 entries.  The test fills the padding
  with NaN sentinels through the raw state, steps every boundary kind and kernel variant at
  ragged sizes, and checks on the host that the sentinels are untouched.  A kernel that read the
  padding would also meet the NaN and raise the divergence flag.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from paper_2410_09739_gb300 import fpclbm as F

pytestmark = pytest.mark.gpu

UINT = {"fp64": np.uint64, "fp32": np.uint32, "fp16": np.uint16, "bf16": np.uint16}
NAN_BITS = {"fp64": 0x7FF8DEADBEEF0001, "fp32": 0x7FC0BEEF, "fp16": 0x7E55, "bf16": 0x7FC5}


def channel(nx, ny, nz, prec, bc=1, tau=0.6, Fx=2e-5, seed=3):
    lat = F.Lattice(nx, ny, nz, prec, bc)
    lat.set_params(tau)
    if bc in (0, 1, 3):
        lat.set_force(Fx, 0, 0)
    lat.init_fields(*W.channel_fields(nx, ny, nz, 0.01, seed=seed))
    return lat


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16", "bf16"])
@pytest.mark.parametrize("n", [8, 41])
@pytest.mark.parametrize("bc", [0, 1])
def test_resume_from_raw_state_is_bit_identical(prec, n, bc):
    nx, ny, nz = 24, 10, 6
    with channel(nx, ny, nz, prec, bc) as a:
        a.step(n)
        raw, k = a.get_state()
        assert k == n and raw.size == F.fpclbm_state_bytes(a.h)
        a.step(n)
        end_a, ka = a.get_state()
    with F.Lattice(nx, ny, nz, prec, bc) as b:
        b.set_params(0.6)
        if bc in (0, 1):
            b.set_force(2e-5, 0, 0)
        b.set_state(raw, k)
        assert b.step_count() == n
        b.step(n)
        end_b, kb = b.get_state()
    assert ka == kb == 2 * n
    assert np.array_equal(end_a, end_b)


def test_resume_ensemble_from_raw_state_is_bit_identical():
    sides = [8, 12, 16]
    taus = [0.55, 0.6, 0.7]
    dims = [(s, s, s) for s in sides]
    flds = W.ensemble_fields(sides, seed=4)
    flat = [np.concatenate([np.asarray(f[q]).reshape(-1) for f in flds]) for q in range(4)]

    def make():
        lat = F.Lattice.ensemble(dims, taus, "fp32")
        lat.set_params(1.0)
        return lat

    with make() as a:
        a.init_fields(*flat)
        a.step(7)
        raw, k = a.get_state()
        a.step(7)
        end_a, _ = a.get_state()
    with make() as b:
        b.set_state(raw, k)
        b.step(7)
        end_b, _ = b.get_state()
    assert np.array_equal(end_a, end_b)


def test_set_state_rejects_a_wrong_size_or_step_count():
    with channel(8, 6, 4, "fp32") as lat:
        raw, k = lat.get_state()
        for bad_raw, bad_k in ((raw[:-1], k), (np.concatenate([raw, raw[:16]]), k), (raw, -1)):
            with pytest.raises(F.FpclbmError) as e:
                lat.set_state(bad_raw, bad_k)
            assert e.value.code == F.FPCLBM_ERR_ARG


def _inject_until_success(make, base):
    """Fail the k-th allocation of make() for k = 0, 1, ...: each must raise ERR_ALLOC and free
    everything; returns the number of allocations make() performs."""
    for k in range(64):
        F.fpclbm_test_alloc_hook(k)
        try:
            obj = make()
        except F.FpclbmError as e:
            F.fpclbm_test_alloc_hook(-1)
            assert e.code == F.FPCLBM_ERR_ALLOC, (k, e)
            assert F.fpclbm_test_alloc_hook() == base, k
            continue
        F.fpclbm_test_alloc_hook(-1)
        obj.close()
        assert F.fpclbm_test_alloc_hook() == base
        return k
    raise AssertionError("make() never succeeded")


def test_injected_allocation_failures_leak_nothing_and_leave_the_library_usable():
    F.fpclbm_test_alloc_hook(-1)
    base = F.fpclbm_test_alloc_hook()
    n1 = _inject_until_success(lambda: F.Lattice(40, 24, 18, "fp32", 1), base)
    n2 = _inject_until_success(lambda: F.Lattice.ensemble([(8, 8, 8), (12, 12, 12)], [0.6, 0.7], "fp32"), base)
    n3 = _inject_until_success(lambda: F.Lattice2D(32, 24, "fp32"), base)
    assert n1 >= 6 and n2 >= n1 + 2 and n3 >= 3  # every allocation of each create path was failed once
    # the next handle works
    with channel(16, 8, 8, "fp32") as lat:
        lat.step(5)
        d = lat.diagnostics()
        assert np.all(np.isfinite(d))
    assert F.fpclbm_test_alloc_hook() == base


def test_injected_allocation_failure_in_training_scratch():
    torch = pytest.importorskip("torch")
    F.fpclbm_test_alloc_hook(-1)
    base = F.fpclbm_test_alloc_hook()
    rng = np.random.default_rng(1)
    X = torch.from_numpy(rng.normal(size=(512, 9)).astype(np.float32)).cuda()
    T = torch.from_numpy(rng.normal(size=512).astype(np.float32) * 0.01).cuda()
    failed = 0
    for k in range(16):
        F.fpclbm_test_alloc_hook(k)
        try:
            F.fpclbm_closure_train(X, T, 512, 1, 64, 1e-3, seed=1)
        except F.FpclbmError as e:
            F.fpclbm_test_alloc_hook(-1)
            assert e.code == F.FPCLBM_ERR_ALLOC
            assert F.fpclbm_test_alloc_hook() == base
            failed += 1
            continue
        F.fpclbm_test_alloc_hook(-1)
        break
    assert failed >= 2
    assert F.fpclbm_test_alloc_hook() == base


def _padding_views(raw, prec, boxes):
    """The padding entries [n_b, stride_b) of every slot row of every box, as integer views."""
    u = raw.view(UINT[prec])
    out, off = [], 0
    for n in boxes:
        stride = (n + 63) // 64 * 64
        for s in range(27):
            out.append(u[off + s * stride + n: off + (s + 1) * stride])
        off += 27 * stride
    return out


def _check_guard_bands(lat, prec, boxes, steps):
    raw, k = lat.get_state()
    pads = _padding_views(raw, prec, boxes)
    assert sum(p.size for p in pads) > 0
    for p in pads:
        p[:] = NAN_BITS[prec]
    lat.set_state(raw, k)
    lat.step(steps)  # raises DIVERGED if a kernel read a NaN sentinel
    assert np.all(np.isfinite(lat.diagnostics()))
    after, _ = lat.get_state()
    for p in _padding_views(after, prec, boxes):
        assert np.all(p == UINT[prec](NAN_BITS[prec]))


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16", "bf16"])
@pytest.mark.parametrize("bc,lid", [(0, 0.0), (1, 0.0), (1, 0.02), (2, 0.02), (3, 0.0)])
@pytest.mark.parametrize("launch", ["128:2:0", "128:2:2", "128:2:3"])
@pytest.mark.parametrize("shape", [(7, 5, 3), (16, 5, 3)])
def test_guard_bands_untouched(monkeypatch, prec, bc, lid, launch, shape):
    monkeypatch.setenv("FPCLBM_LAUNCH", launch)
    nx, ny, nz = shape
    with F.Lattice(nx, ny, nz, prec, bc) as lat:
        lat.set_params(0.7, 0.2)
        if lid:
            lat.set_wall_velocity(lid)
        elif bc != 2:
            lat.set_force(1e-5, 0, 0)
        lat.init_fields(*W.channel_fields(nx, ny, nz, 0.01, seed=9))
        _check_guard_bands(lat, prec, [nx * ny * nz], 37)


def test_guard_bands_untouched_ensemble():
    sides = [5, 7, 9]
    dims = [(s, s, s) for s in sides]
    flds = W.ensemble_fields(sides, seed=5)
    flat = [np.concatenate([np.asarray(f[q]).reshape(-1) for f in flds]) for q in range(4)]
    with F.Lattice.ensemble(dims, [0.55, 0.6, 0.7], "fp32") as lat:
        lat.set_params(1.0)
        lat.init_fields(*flat)
        _check_guard_bands(lat, "fp32", [s ** 3 for s in sides], 37)
