"""The host packing of the learned closure's weights (fpclbm_closure_pack: the words
fpclbm_set_closure uploads) read back the way the fused inference reads them, without a GPU.

A numpy model of one warp's mma.sync.m16n8k16 operands (PTX fragment layout for bf16: lane =
4 g + t; A registers a0..a3 hold rows g, g+8 and columns 2t, 2t+1 and 2t+8, 2t+9; B registers
b0, b1 hold k = 2t, 2t+1 and 2t+8, 2t+9 of column n = g; C holds rows g, g+8 and columns 2t, 2t+1)
gathers each layer's B matrix from the packed words, forms the layer-1 A fragments from the
inputs the way the kernel does (the bias input 1 in column 9), re-packs the layer-1 accumulators as
layer-2 A fragments, adds b2 through the constant-1 K tile, and must reproduce the MLP of the
oracle with the same bf16 roundings of the inputs and the first hidden layer for the 32 cells of a
warp.  A mistake in the packing (a transposed block, a wrong k offset, b1 or b2 in the wrong slot)
or in the fragment bookkeeping changes the output by far more than the tolerance.
"""
import numpy as np
import pytest

from oracle import closure as C
from paper_2410_09739_gb300 import fpclbm as F

CP_F1, CP_F2, CP_B1, CP_B2, CP_W3, CP_B3, CP_F2B, CP_WORDS = 0, 512, 2560, 2624, 2688, 2752, 2756, 3012


def bf16_round(x):
    a = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    bits = ((a + ((a >> 16) & 1) + 0x7FFF) >> 16).astype(np.uint16)
    return (bits.astype(np.uint32) << 16).view(np.float32).astype(np.float64), bits


def halves(word):
    """The two bf16 values of a 32-bit word (low half first)."""
    w = np.uint32(word)
    lo = np.array([np.uint32(w & 0xFFFF) << 16], dtype=np.uint32).view(np.float32)[0]
    hi = np.array([np.uint32(w & 0xFFFF0000)], dtype=np.uint32).view(np.float32)[0]
    return float(lo), float(hi)


def f32(word):
    return float(np.array([word], dtype=np.uint32).view(np.float32)[0])


def b_matrix(words0, words1):
    """16 x 8 B operand from the per-lane registers b0 (k = 2t, 2t+1) and b1 (k = 2t+8, 2t+9)."""
    B = np.zeros((16, 8))
    for lane in range(32):
        g, t = lane // 4, lane % 4
        B[2 * t, g], B[2 * t + 1, g] = halves(words0[lane])
        B[2 * t + 8, g], B[2 * t + 9, g] = halves(words1[lane])
    return B


def a_matrix(regs):
    """16 x 16 A operand from per-lane registers (a0, a1, a2, a3), each a pair of values."""
    A = np.zeros((16, 16))
    for lane in range(32):
        g, t = lane // 4, lane % 4
        a0, a1, a2, a3 = regs[lane]
        A[g, 2 * t:2 * t + 2] = a0
        A[g + 8, 2 * t:2 * t + 2] = a1
        A[g, 2 * t + 8:2 * t + 10] = a2
        A[g + 8, 2 * t + 8:2 * t + 10] = a3
    return A


def c_fragments(D):
    """Per-lane accumulator registers (c0, c1, c2, c3) of a 16 x 8 product D."""
    return [(D[l // 4, 2 * (l % 4)], D[l // 4, 2 * (l % 4) + 1], D[l // 4 + 8, 2 * (l % 4)],
             D[l // 4 + 8, 2 * (l % 4) + 1]) for l in range(32)]


def warp_network(P, X):
    """delta omega of the 32 cells of a warp (rows of X) from the packed words P."""
    xin = np.zeros((32, 16))
    xin[:, :9], _ = bf16_round(X)
    xin[:, 9] = 1.0  # input 9: the constant 1 that carries b1
    out = np.zeros(32)
    for mt in range(2):
        rows = xin[16 * mt:16 * mt + 16]
        # layer-1 A fragments as the kernel gathers them: a0/a1 the pair t of rows g / g+8, a2/a3
        # the pair (x8, 1) for t = 0 and zeros otherwise
        regs1 = []
        for lane in range(32):
            g, t = lane // 4, lane % 4
            a0, a1 = rows[g, 2 * t:2 * t + 2], rows[g + 8, 2 * t:2 * t + 2]
            a2 = rows[g, 8:10] if t == 0 else np.zeros(2)
            a3 = rows[g + 8, 8:10] if t == 0 else np.zeros(2)
            regs1.append((a0, a1, a2, a3))
        A1 = a_matrix(regs1)
        # layer 1 + tanh; the accumulator of n-tile nt becomes A2[kt = nt // 2][(nt % 2) * 2 + {0, 1}]
        A2 = [[[None] * 4 for _ in range(4)] for _ in range(32)]
        for nt in range(8):
            B = b_matrix(P[CP_F1 + nt * 64:CP_F1 + nt * 64 + 64:2], P[CP_F1 + nt * 64 + 1:CP_F1 + nt * 64 + 64:2])
            cf = c_fragments(A1 @ B)
            for lane in range(32):
                c0, c1, c2, c3 = cf[lane]
                h = (nt % 2) * 2
                A2[lane][nt // 2][h] = bf16_round(np.tanh([c0, c1]))[0]
                A2[lane][nt // 2][h + 1] = bf16_round(np.tanh([c2, c3]))[0]
        # the constant-1 A fragment of layer 2's bias tile: (1, 0) in a0 and a1 of lanes with t = 0
        ones = [np.array([1.0, 0.0]) if l % 4 == 0 else np.zeros(2) for l in range(32)]
        Aone = a_matrix([(ones[l], ones[l], np.zeros(2), np.zeros(2)) for l in range(32)])
        y = np.zeros(16)
        for nt in range(8):
            wb = P[CP_F2B + nt * 32:CP_F2B + nt * 32 + 32]
            Z = Aone @ b_matrix(wb, np.zeros(32, dtype=np.uint32))  # b2 through the constant-1 tile
            for kt in range(4):
                base = CP_F2 + (nt * 4 + kt) * 64
                Ak = a_matrix([(A2[l][kt][0], A2[l][kt][1], A2[l][kt][2], A2[l][kt][3]) for l in range(32)])
                Z = Z + Ak @ b_matrix(P[base:base + 64:2], P[base + 1:base + 64:2])
            w3 = np.array([f32(P[CP_W3 + 8 * nt + j]) for j in range(8)])
            y += np.tanh(Z) @ w3
        out[16 * mt:16 * mt + 16] = y + f32(P[CP_B3])
    return out


def mlp_bf16_operands(theta, X):
    p = C.unpack(theta)
    xb, _ = bf16_round(X)
    h1, _ = bf16_round(np.tanh(xb @ p["W1"].T + p["b1"]))
    h2 = np.tanh(h1 @ p["W2"].T + p["b2"])
    return h2 @ p["W3"][0] + p["b3"][0]


@pytest.mark.parametrize("seed", [1, 2])
def test_packed_closure_evaluates_the_oracle_mlp(seed):
    rng = np.random.default_rng(seed)
    th = C.init_params(seed) * 3.0
    th[576:640] = rng.uniform(-0.5, 0.5, 64)    # b1
    th[4736:4800] = rng.uniform(-0.5, 0.5, 64)  # b2
    th[-65:-1] = rng.uniform(-0.2, 0.2, 64)     # W3
    th[-1] = -0.05                              # b3
    wv, wbits = bf16_round(th)
    P = F.fpclbm_closure_pack(wbits)
    assert P.shape == (CP_WORDS,) and P.dtype == np.uint32
    # the fp32 copies of the biases and output layer are the bf16 values widened
    p = C.unpack(wv)
    assert np.array_equal(P[CP_B1:CP_B1 + 64].view(np.float32).astype(np.float64), p["b1"])
    assert np.array_equal(P[CP_B2:CP_B2 + 64].view(np.float32).astype(np.float64), p["b2"])
    assert np.array_equal(P[CP_W3:CP_W3 + 64].view(np.float32).astype(np.float64), p["W3"][0])
    assert np.all(P[CP_B3 + 1:CP_F2B] == 0)
    X = np.concatenate([rng.normal(scale=0.5, size=(32, 6)), rng.normal(scale=0.5, size=(32, 3))], axis=1)
    got = warp_network(P, X)
    ref = mlp_bf16_operands(wv, X)
    assert np.max(np.abs(got - ref)) <= 1e-9 * (1 + np.max(np.abs(ref)))
    assert np.std(ref) > 1e-3  # the network's output varies across the cells


def test_closure_pack_rejects_wrong_sizes():
    _, wbits = bf16_round(C.init_params(3))
    with pytest.raises(F.FpclbmError):
        F.fpclbm_closure_pack(wbits[:-1])
