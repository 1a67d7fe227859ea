"""Learned closure on the GPU: training data (filter + labels), training gradients, inference.

Tolerances: sampled features/labels are fp64 on the device and rounded to
float32 on output (relative 2^-24, checked at 1e-5 of each column's scale);
gradients of the bf16-weight fp32 kernels against the fp64 oracle with the
same bf16 weights: relative 2-norm per tensor <= 2e-2 (the stated bound;
fp32 summation of ~64-term sums gives ~1e-6); inference (tensor-core MLP with
bf16 operands): the oracle-side network takes the same bf16 roundings of its
inputs and first hidden layer, and one step is checked at 1e-6 absolute like
every fp32 path.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from oracle import closure as C
from paper_2410_09739_gb300 import fpclbm as F

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def bf16_round(x):
    """Round-to-nearest-even to bf16, returned as (float64 values, uint16 bits)."""
    a = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    bias = ((a >> 16) & 1) + 0x7FFF
    bits = ((a + bias) >> 16).astype(np.uint16)
    vals = (bits.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    return vals, bits


@pytest.mark.parametrize("walls", [0, 1])
def test_sample_matches_oracle_filter(walls):
    nx, ny, nz, r = 16, 12, 8, 4
    tau_c = 0.52
    rho, ux, uy, uz = W.random_fields(nx, ny, nz, seed=30 + walls, u_amp=0.05)
    with F.Lattice(nx, ny, nz, "fp32", walls) as lat:
        lat.set_params(0.7)
        lat.set_force(1e-5, 0, 0)
        lat.init_fields(rho, ux, uy, uz)
        lat.step(3)
        nc = (nx // r) * (ny // r) * (nz // r)
        X = np.zeros((nc, 9), np.float32)
        T = np.zeros(nc, np.float32)
        F.fpclbm_closure_sample(lat.h, r, tau_c, X, T)
        f = lat.get_populations()
    R, A, B, Cz = O.moments(f, (1e-5, 0, 0))
    Xr, Tr = C.sample(R, A, B, Cz, r, tau_c, bool(walls))
    for k in range(9):
        scale = np.max(np.abs(Xr[:, k])) + 1e-30
        assert np.max(np.abs(X[:, k] - Xr[:, k])) <= 1e-5 * scale, k
    assert np.max(np.abs(T - Tr)) <= 1e-5 * (np.max(np.abs(Tr)) + 1e-30)
    assert np.any(Tr < 0)  # some cells carry an eddy viscosity


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def _loss_and_grad_bf16_operands(theta, X, t):
    """The training kernel's arithmetic: the operands of its tensor-core products (inputs x, first
    hidden layer H1, and the back-propagated G2 = dL/dZ2 and G1 = dL/dZ1) rounded to bf16, products
    exact here (fp32 accumulation on the GPU), tanh, the output layer, dL/dy and dw3 unrounded."""
    p = C.unpack(theta)
    n = X.shape[0]
    xb, _ = bf16_round(X)
    h1 = np.tanh(xb @ p["W1"].T + p["b1"])
    h1b, _ = bf16_round(h1)
    h2 = np.tanh(h1b @ p["W2"].T + p["b2"])
    e = h2 @ p["W3"][0] + p["b3"][0] - t
    gy = 2.0 / n * e
    g2b, _ = bf16_round(gy[:, None] * p["W3"][0][None, :] * (1.0 - h2 * h2))
    g1b, _ = bf16_round((g2b @ p["W2"]) * (1.0 - h1 * h1))
    grads = {"W1": g1b.T @ xb, "b1": g1b.sum(0), "W2": g2b.T @ h1b, "b2": g2b.sum(0),
             "W3": (gy @ h2)[None, :], "b3": np.array([gy.sum()])}
    return float(np.mean(e * e)), grads


@pytest.mark.parametrize("n", [1, 64, 200, 1000])
def test_training_gradients_match_fp64_oracle(n):
    """The training kernel's products are bf16 x bf16 -> fp32 tensor-core tiles (x, H1 and the
    back-propagated G2, G1 rounded to bf16).  Against the exact fp64 oracle with the same bf16
    weights the gradients meet the stated bound (relative 2-norm <= 2e-2 per tensor); against the
    same arithmetic with those bf16 roundings they agree to fp32 accumulation (<= 1e-3: a bf16
    rounding of an fp32-accumulated value can differ by one unit from that of the exact value)."""
    rng = np.random.default_rng(n)
    th = C.init_params(n)
    th[C.N_PARAMS - 65:C.N_PARAMS - 1] = rng.uniform(-0.3, 0.3, 64)  # non-zero last layer
    wv, wbits = bf16_round(th)
    X = np.concatenate([rng.normal(scale=0.5, size=(n, 6)), rng.normal(scale=0.5, size=(n, 3))], axis=1)
    X = X.astype(np.float32)
    t = rng.normal(scale=0.3, size=n).astype(np.float32)
    loss, g = F.fpclbm_closure_grad(torch.from_numpy(X).cuda(), torch.from_numpy(t).cuda(), n, wbits)
    L, gr = C.loss_and_grad(wv, X.astype(np.float64), t.astype(np.float64))
    assert abs(loss - L) <= 2e-2 * L
    pg, pr = C.unpack(g.astype(np.float64)), C.unpack(gr)
    Lb, pb = _loss_and_grad_bf16_operands(wv, X.astype(np.float64), t.astype(np.float64))
    assert abs(loss - Lb) <= 1e-5 * Lb
    for name, _ in C.SHAPES:
        assert _rel(pg[name], pr[name]) <= 2e-2, name
        assert _rel(pg[name], pb[name].reshape(pg[name].shape)) <= 1e-3, name


def test_training_is_deterministic():
    """Block gradients are summed in a fixed order (no atomics): two trainings from the same seed
    give the same weights bit for bit."""
    n = 3000
    rng = np.random.default_rng(8)
    X = torch.from_numpy(rng.normal(scale=0.3, size=(n, 9)).astype(np.float32)).cuda()
    t = torch.from_numpy((0.01 * rng.normal(size=n)).astype(np.float32)).cuda()
    w1, l1 = F.fpclbm_closure_train(X, t, n, 3, 256, 1e-3, seed=4)
    w2, l2 = F.fpclbm_closure_train(X, t, n, 3, 256, 1e-3, seed=4)
    assert np.array_equal(w1, w2) and np.array_equal(l1, l2)


def test_training_fits_a_smooth_target():
    n = 20000
    rng = np.random.default_rng(5)
    X = np.concatenate([rng.normal(scale=1e-3, size=(n, 6)), rng.normal(scale=0.05, size=(n, 3))], axis=1)
    t = -0.02 * np.tanh(800.0 * X[:, 3]) ** 2 - 0.5 * X[:, 6] ** 2
    Xd = torch.from_numpy(X.astype(np.float32)).cuda()
    td = torch.from_numpy(t.astype(np.float32)).cuda()
    w, losses = F.fpclbm_closure_train(Xd, td, n, epochs=30, batch=512, lr=3e-3, seed=1)
    assert losses[-1] < 0.05 * losses[0]
    # the folded raw-unit weights reproduce the target through the fp64 oracle
    wv = (w.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    y, _ = C.forward(wv, X)
    assert np.sqrt(np.mean((y - t) ** 2)) < 0.25 * np.std(t)


def _mlp_bf16_operands(theta, x):
    """The inference arithmetic of the fused kernel: bf16 operands (inputs and first hidden layer),
    products accumulated exactly here (fp32 on the GPU), tanh exact here (MUFU on the GPU)."""
    p = C.unpack(theta)
    xb, _ = bf16_round(x)
    h1, _ = bf16_round(np.tanh(p["W1"] @ xb + p["b1"]))
    h2 = np.tanh(p["W2"] @ h1 + p["b2"])
    return float(p["W3"][0] @ h2 + p["b3"][0])


def _learned_step_oracle(f0, theta, omega_base, bc=0):
    """One step of the learned-mode collision with the oracle: per cell, delta omega from the MLP
    on (kappa_2 - kappa_2^Mv, u); the shear rates become max(omega + min(delta omega, 0), 0.02) (the
    correction only adds viscosity, as its training labels do); then collide and push-stream."""
    _, nz, ny, nx = f0.shape
    e = O.velocity_set()
    mnp = [tuple(v) for v in O.moment_exponents()]
    out = np.zeros_like(f0)
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                f = f0[:, z, y, x]
                rho = f.sum()
                u = (f @ e) / rho
                k = O.central_matrix(u) @ f
                K = lambda s: k[mnp.index(s)]  # noqa: E731
                feat = np.array([K((2, 0, 0)) - rho / 3, K((0, 2, 0)) - rho / 3, K((0, 0, 2)) - rho / 3,
                                 K((1, 1, 0)), K((1, 0, 1)), K((0, 1, 1)), u[0], u[1], u[2]])
                dw = _mlp_bf16_operands(theta, feat)
                om = omega_base.copy()
                for j in (4, 5, 6, 8, 9):
                    om[j] = max(om[j] + min(dw, 0.0), 0.02)
                ft = O.collide(f, (0, 0, 0), om, O.EQ_MODE_FP)
                for a in range(27):
                    out[a, (z + e[a, 2]) % nz, (y + e[a, 1]) % ny, (x + e[a, 0]) % nx] = ft[a]
    return out


def test_learned_inference_matches_oracle():
    """60 cells: one full warp and a ragged tail warp.  Network with the output scale of a trained
    closure (|delta omega| ~ 5e-2).  Both sides round the inputs and the first hidden layer to bf16;
    what remains is the MUFU tanh (absolute ~2^-11 per activation): |d delta omega| <~ 64 * 0.05 *
    5e-4 = 1.6e-3 at worst, and one step moves by ~9e-8 per 1e-4 of delta omega here, so <= 1e-6
    holds with margin while the closure itself moves the step by ~5e-5."""
    nx, ny, nz = 5, 4, 3
    rng = np.random.default_rng(9)
    th = C.init_params(3) * 3.0
    th[-65:-1] = rng.uniform(-0.05, 0.05, 64)
    th[-1] = -0.05
    wv, wbits = bf16_round(th)
    rho, ux, uy, uz = W.random_fields(nx, ny, nz, seed=4, u_amp=0.05)
    f0 = O.init_equilibrium(rho, ux, uy, uz) * (1 + 0.02 * rng.uniform(-1, 1, (27, nz, ny, nx)))
    tau = 0.7
    with F.Lattice(nx, ny, nz, "fp32") as lat:
        lat.set_closure(wbits)
        lat.set_params(tau, 0.0, F.FPCLBM_DIFF_FP_LEARNED)
        lat.set_populations(f0)
        fq = lat.get_populations()
        lat.step(1)
        got = lat.get_populations()
    ref = _learned_step_oracle(fq, wv, O.rates(tau))
    assert np.max(np.abs(got - ref)) <= 1e-6
    plain = O.step(fq, omega=O.rates(tau))
    assert np.max(np.abs(ref - plain)) > 1e-5  # the closure changed the step


@pytest.mark.parametrize("launch", ["128:2:0", "128:2:2"])
@pytest.mark.parametrize("drift", [0.0, 0.3])
@pytest.mark.parametrize("shape", [(5, 4, 3), (8, 6, 5)])
def test_learned_step_variants_match_oracle(monkeypatch, launch, drift, shape):
    """The learned mode in both kernel variants (one cell per thread; two cells per thread with the
    MLP run once per lane of the pair) and both rate settings (unit rates of orders 3-6, whose
    moments are set to their attractors, and the order-scaled rates k * drift), over two steps
    (both AA parities).  60 cells leave tail lanes in the warp-collective MLP; 240 cells with even
    nx take the neighbouring-cell odd step.  Same 1e-6 per step as the one-step test."""
    monkeypatch.setenv("FPCLBM_LAUNCH", launch)
    nx, ny, nz = shape
    rng = np.random.default_rng(19 + nx)
    th = C.init_params(4) * 3.0
    th[-65:-1] = rng.uniform(-0.05, 0.05, 64)
    th[-1] = -0.05
    wv, wbits = bf16_round(th)
    rho, ux, uy, uz = W.random_fields(nx, ny, nz, seed=6, u_amp=0.05)
    f0 = O.init_equilibrium(rho, ux, uy, uz) * (1 + 0.02 * rng.uniform(-1, 1, (27, nz, ny, nx)))
    tau = 0.7
    with F.Lattice(nx, ny, nz, "fp32") as lat:
        lat.set_closure(wbits)
        lat.set_params(tau, drift, F.FPCLBM_DIFF_FP_LEARNED)
        lat.set_populations(f0)
        fq = lat.get_populations()
        ref = fq
        for n in (1, 2):
            lat.step(1)
            got = lat.get_populations()
            ref = _learned_step_oracle(ref, wv, O.rates(tau, drift))
            assert np.max(np.abs(got - ref)) <= 1e-6 * n, n
        lau = lat.launch()
    assert lau["variant"] == int(launch[-1])
    assert lau["mode"] == (6 if drift == 0.0 else 2)
