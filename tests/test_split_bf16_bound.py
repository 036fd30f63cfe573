"""The error level of the split-BF16 products of the tensor-core z solve (reading R21), on
the CPU: every operand x held as hi = bf16(x), lo = bf16(x - hi) and the product formed as
Ahi Bhi + Alo Bhi + Ahi Blo.  Emulated here in FP64 arithmetic (so that only the splitting
is measured): the 16 significant bits of hi + lo and the dropped Alo Blo term give a
transform error below 2^-17 of the column's largest value (about 4e-6 here), and the full
solve D^T diag(1/sigma) D stays within 2e-5 (the GPU kernel measured 0.6-1.8e-5 against an
FP64 dense solve); a 2-term product (Ahi Bhi only) is worse by a factor of about 500."""
import numpy as np


def bf16(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def split(x):
    x32 = np.asarray(x, dtype=np.float32).astype(np.float64)
    hi = bf16(x32)
    lo = bf16(x32 - hi)
    return hi, lo


def dct2(n):
    m = np.arange(n)[:, None]
    z = np.arange(n)[None, :]
    c = np.where(m == 0, np.sqrt(1.0 / n), np.sqrt(2.0 / n))
    return c * np.cos(np.pi * m * (2 * z + 1) / (2 * n))


def test_bf16_rounding_by_hand():
    assert bf16(1.0) == 1.0
    assert bf16(1.0 + 2.0 ** -8) == 1.0                  # a tie rounds to even
    assert bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6  # the other tie rounds up to even
    hi, lo = split(np.float32(np.pi))
    assert abs(hi + lo - np.float32(np.pi)) <= 2.0 ** -16 * np.pi


def test_split_products_and_solve_within_the_stated_bounds():
    rng = np.random.default_rng(350)
    for n in (128, 256):
        D = dct2(n)
        X = rng.uniform(-1.0, 1.0, (n, 96)).astype(np.float32).astype(np.float64)
        Dh, Dl = split(D)
        Xh, Xl = split(X)
        exact = D @ X
        three = Dh @ Xh + Dl @ Xh + Dh @ Xl
        two = Dh @ Xh
        rel3 = np.abs(three - exact).max() / np.abs(exact).max()
        rel2 = np.abs(two - exact).max() / np.abs(exact).max()
        assert rel3 <= 2.0 ** -17, rel3
        assert rel2 > 100 * rel3
        # the Poisson-type solve: x <- D^T diag(1/L) D x with the eigenvalues of the
        # zero-gradient second difference plus a periodic part (no zero mode here)
        h = 1.0 / n
        lam = -(4.0 / h ** 2) * np.sin(np.pi * np.arange(n) / (2 * n)) ** 2 - 40.0
        Y = np.diag(1.0 / lam) @ three
        Yh, Yl = split(Y)
        sol3 = Dh.T @ Yh + Dl.T @ Yh + Dh.T @ Yl
        sol = D.T @ np.diag(1.0 / lam) @ D @ X
        rel = np.abs(sol3 - sol).max() / np.abs(sol).max()
        assert rel <= 2e-5, rel
