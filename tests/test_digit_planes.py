"""CPU checks of the digit-plane scheme behind the FP64-class tensor-core
products (csrc/oz_gemm.cu), emulated in numpy with the kernel's float32
steps: the exactness bound of the diagonal sums, the error-free digit
extraction of float-float values, and the product error against FP64."""
import numpy as np

L, BITS = 8, 7


def digits_ff(h, l, F):
    """The kernel's extraction: v = (h + l) 2^-F; per plane v <- 128 v,
    digit = rint(high part), high part keeps the remainder, (high, low)
    renormalised by TwoSum.  All in float32."""
    f32 = np.float32
    vh = np.ldexp(h.astype(f32), -F).astype(f32)
    vl = np.ldexp(l.astype(f32), -F).astype(f32)
    out = []
    for _ in range(L):
        vh = (vh * f32(128)).astype(f32)
        vl = (vl * f32(128)).astype(f32)
        q = np.rint(vh).astype(f32)
        vh = (vh - q).astype(f32)
        s = (vh + vl).astype(f32)
        bb = (s - vh).astype(f32)
        e = ((vh - (s - bb)).astype(f32) + (vl - bb).astype(f32)).astype(f32)
        vh, vl = s, e
        out.append(q.astype(np.float64))
    return np.array(out)


def digits_fp64(a, E):
    v = np.ldexp(a, -E)
    out = []
    for _ in range(L):
        v = v * 128.0
        q = np.rint(v)
        v = v - q
        out.append(q)
    return np.array(out)


def test_diagonal_sums_stay_exact_below_k_409():
    """Diagonal d holds the pairs s + t = d: at most two with a first-plane
    digit (|digit| <= 128 against <= 64) and d - 1 of later planes (64 x 64);
    summed over K the bound stays below 2^24 (exact in FP32) for K <= 409."""
    for d in range(L):
        pairs = [(s, d - s) for s in range(d + 1) if s < L and d - s < L]
        bound = sum((128 if s == 0 else 64) * (128 if t == 0 else 64) for s, t in pairs)
        assert bound * 409 < 2 ** 24, (d, bound)
        if d >= 1:
            assert bound == 2 ** 12 * (d + 3)


def test_ff_digits_are_bf16_exact_and_reconstruct():
    rng = np.random.default_rng(7)
    x = rng.standard_normal(4000) * np.exp2(rng.integers(-40, 40, 4000))
    h = x.astype(np.float32)
    l = (x - h.astype(np.float64)).astype(np.float32)
    F = int(np.frexp(np.abs(h).max())[1])
    d = digits_ff(h, l, F)
    assert np.abs(d[0]).max() <= 128 and np.abs(d[1:]).max() <= 64
    # integers of at most 8 significant bits: exact in bf16
    assert np.all(d == np.rint(d))
    rec = sum(d[t] * 2.0 ** (-7 * (t + 1)) for t in range(L)) * 2.0 ** F
    ff = h.astype(np.float64) + l.astype(np.float64)
    assert np.max(np.abs(rec - ff)) <= 2.0 ** (F - 56)


def test_emulated_product_matches_fp64():
    """Rows of A with their own scales, panel columns over 2^-60 .. 2^60:
    the diagonal sums (exact), combined with the row and column exponents,
    against the FP64 product of the FP64 A and the float-float panel."""
    rng = np.random.default_rng(11)
    N, ncol = 96, 40
    A = rng.standard_normal((N, N)) * np.exp2(rng.uniform(-8, 8, (N, 1)))
    B = rng.standard_normal((N, ncol)) * np.exp2(np.linspace(-60, 60, ncol))[None, :]
    Bh = B.astype(np.float32)
    Bl = (B - Bh.astype(np.float64)).astype(np.float32)
    E = np.array([np.frexp(np.abs(A[i]).max())[1] for i in range(N)])
    F = np.array([np.frexp(np.abs(Bh[:, j]).max())[1] for j in range(ncol)])
    Ad = np.stack([digits_fp64(A[i], E[i]) for i in range(N)], 1)  # [L][N][K]
    Bd = np.stack([digits_ff(Bh[:, j], Bl[:, j], int(F[j])) for j in range(ncol)], 2)  # [L][K][ncol]
    acc = np.zeros((L, N, ncol))
    for s in range(L):
        for t in range(L - s):
            acc[s + t] += Ad[s] @ Bd[t]
    assert np.abs(acc).max() < 2 ** 24
    C = sum(acc[d] * 2.0 ** (-7 * d) for d in range(L)) * np.exp2(E[:, None] + F[None, :] - 14)
    ref = A @ (Bh.astype(np.float64) + Bl.astype(np.float64))
    scale = np.abs(A) @ np.abs(Bh.astype(np.float64))
    assert np.max(np.abs(C - ref) / scale) < 1e-14
