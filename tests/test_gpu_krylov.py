"""The Krylov inner product (sgoc_inner_product) against the exactly rounded sum.

The reference is math.fsum of the float64 products of the operands: a product
of two float32 values is exact in float64, and fsum rounds the exact sum once,
so the reference is the correctly rounded inner product.  Bounds:
* float64 operands (float64 products and sums): |err| <= n * 2^-53 * sum|a b|
  (the textbook bound of recursive summation, any order);
* float32 operands (error-free float32 transformations, leading parts summed in
  float64, small parts in float32): |err| <= 2^-40 * sum|a b|, a margin of 2^8
  over the order-2^-48 analysis, and far below the float32 bound (about n 2^-24).
Both paths (the four-wide kernel for 16-byte-aligned float32 operands and the
scalar kernel otherwise) are checked on lengths with ragged tails, on vectors
with heavy cancellation, and for bitwise reproducibility.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def cuda_ready():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests selected but no CUDA device is visible")
    from paper_2512_23804_gb300 import build
    build.build()


def exact(a, b):
    p = a.astype(np.float64) * b.astype(np.float64)
    return math.fsum(p.tolist()), float(np.abs(p).sum())


@pytest.mark.parametrize("n", [0, 1, 3, 4, 7, 4096, 1_000_003, 4_064_508])
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("offset", [0, 1])
def test_inner_product_against_the_exact_sum(n, dtype, offset):
    from paper_2512_23804_gb300 import abi
    rng = np.random.default_rng(n + offset)
    a = rng.standard_normal(n + offset).astype(dtype)
    b = rng.standard_normal(n + offset).astype(dtype)
    if n > 10:
        b[: n // 2] = -a[: n // 2] * 1.0000001          # heavy cancellation in half of the terms
    ta = torch.from_numpy(a).cuda()[offset:]
    tb = torch.from_numpy(b).cuda()[offset:]
    got = abi.inner_product(ta, tb).item()
    ref, mag = exact(a[offset:], b[offset:])
    bound = (n * 2.0 ** -53 if dtype == np.float64 else 2.0 ** -40) * mag
    assert abs(got - ref) <= bound, (got, ref, bound)
    again = abi.inner_product(ta, tb).item()
    assert again == got                                     # fixed order: bitwise reproducible


def test_float32_inner_product_beats_float32_accumulation():
    """The float32 path is not a float32 sum: on a cancelling sum of 4e6 terms its error is far
    below what float32 accumulation of the same products makes."""
    from paper_2512_23804_gb300 import abi
    rng = np.random.default_rng(5)
    n = 4_000_000
    a = rng.standard_normal(n).astype(np.float32)
    b = (rng.standard_normal(n) * 1e-3).astype(np.float32)
    b[::2] = -a[::2]
    ref, mag = exact(a, b)
    got = abi.inner_product(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()).item()
    f32 = float(torch.dot(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()).item())
    assert abs(got - ref) <= 2.0 ** -40 * mag
    assert abs(got - ref) * 1e3 < max(abs(f32 - ref), 1e-300)
