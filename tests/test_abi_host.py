"""The C-ABI library loads, exports every entry point of include/sgoc.h, and its
host-side set-up (chaos multi-indices, triple-product tables, validation) agrees
with the oracle.  No GPU is needed: nothing here launches device work."""
import ctypes
import os
import re

import numpy as np
import pytest

import sg_inputs as si
from oracle import basis
from paper_2512_23804_gb300 import abi, SGProblem

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built_library():
    from paper_2512_23804_gb300 import build
    build.build()


def header_symbols():
    txt = open(os.path.join(ROOT, "include", "sgoc.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(sgoc_[a-z_0-9]+)\s*\(", txt)))


def test_status_codes_match_header():
    txt = open(os.path.join(ROOT, "include", "sgoc.h")).read()
    codes = {name: int(v) for name, v in re.findall(r"\b(SGOC_(?:OK|ERR_[A-Z_]+))\s*=\s*(\d+)", txt)}
    assert len(codes) == 10
    for name, v in codes.items():
        assert getattr(abi, name) == v, name
        assert abi.STATUS_NAMES[v] == name


def test_exports_every_declared_symbol():
    lib = abi.load()
    syms = header_symbols()
    assert len(syms) >= 15
    for s in syms:
        assert hasattr(lib, s), s
    assert set(syms) == set(abi.SIGNATURES)


@pytest.mark.parametrize("M,p", [(2, 2), (3, 3), (6, 3), (8, 3), (4, 4), (1, 5), (0, 3), (5, 0)])
def test_pc_indices_bit_exact(M, p):
    pr = si.random_small(0, nx=4, M=M, p=p)
    sp = SGProblem.from_problem(pr)
    assert sp.P == basis.multi_indices(M, p).shape[0]
    assert np.array_equal(sp.pc_indices(), basis.multi_indices(M, p))


@pytest.mark.parametrize("M,p", [(2, 2), (3, 3), (6, 3), (2, 4)])
def test_triple_products_match_oracle(M, p):
    pr = si.random_small(0, nx=4, M=M, p=p)
    sp = SGProblem.from_problem(pr)
    k, a, b, c = sp.triple_products()
    G = basis.g_matrices(M, p)
    dense = [np.zeros_like(G[0]) for _ in range(M + 1)]
    for kk, aa, bb, cc in zip(k, a, b, c):
        dense[kk][aa, bb] = cc
    for kk in range(1, M + 1):
        assert np.array_equal(dense[kk] != 0, G[kk] != 0)          # pattern bit-exact
        assert np.max(np.abs(dense[kk] - G[kk])) <= 1e-15
    # sorted by k inside each output column (the kernel relies on it)
    for bb in np.unique(b):
        ks = k[b == bb]
        assert np.all(np.diff(ks) >= 0)


def test_sizes():
    pr = si.time_problem(8, 2, 2, 0.5, 0.3, 1e-2, 3)
    sp = SGProblem.from_problem(pr)
    assert (sp.n, sp.P, sp.slabs, sp.kkt_size) == (49, 6, 3, 3 * 3 * 6 * 49)
    assert sp.persistent_bytes > 0 and sp.workspace_bytes > sp.kkt_size * 8


def _create(**over):
    pr = si.random_small(0, nx=8, M=2, p=2)
    args = dict(nx=pr.nx, M=pr.M, p=pr.p, kappa=pr.kappa, beta=pr.beta, yhat=pr.yhat)
    args.update(over)
    return SGProblem(**args)


@pytest.mark.parametrize("over,status", [
    (dict(nx=12, kappa=np.ones((3, 12, 12)), yhat=np.zeros((1, 121))), "SGOC_ERR_UNSUPPORTED"),
    (dict(nx=1, kappa=np.ones((3, 1, 1)), yhat=np.zeros((1, 1))), "SGOC_ERR_INVALID_ARG"),
    (dict(beta=0.0), "SGOC_ERR_INVALID_ARG"),
    (dict(beta=-1.0), "SGOC_ERR_INVALID_ARG"),
    (dict(r=5), "SGOC_ERR_INVALID_ARG"),
    (dict(M=17, kappa=np.ones((18, 8, 8))), "SGOC_ERR_INVALID_ARG"),
    (dict(cheb_steps=0), "SGOC_ERR_INVALID_ARG"),
    (dict(omega=2.5), "SGOC_ERR_INVALID_ARG"),
])
def test_invalid_problems_rejected(over, status):
    with pytest.raises(abi.SgocError) as ei:
        _create(**over)
    assert abi.STATUS_NAMES[ei.value.status] == status


def test_exact_mean_solve_option_scope():
    """mean_solve = "exact" (the tensor-core fast-diagonalisation solve) exists for mixed
    precision on 64 x 64 and 128 x 128 grids; float64 and other grids are refused at set-up."""
    for nx, precision, ok in [(64, "mixed", True), (128, "mixed", True), (32, "mixed", False),
                              (256, "mixed", False), (64, "fp64", False)]:
        pr = si.random_small(7, nx=nx, M=1, p=1)
        if ok:
            sp = SGProblem.from_problem(pr, precision=precision, mean_solve="exact")
            assert sp.persistent_bytes > SGProblem.from_problem(pr, precision=precision).persistent_bytes
        else:
            with pytest.raises(abi.SgocError) as ei:
                SGProblem.from_problem(pr, precision=precision, mean_solve="exact")
            assert abi.STATUS_NAMES[ei.value.status] == "SGOC_ERR_UNSUPPORTED"


def test_nonconstant_mean_and_nan_rejected():
    pr = si.random_small(0, nx=8, M=2, p=2)
    k = pr.kappa.copy()
    k[0, 3, 3] = 1.5
    with pytest.raises(abi.SgocError) as ei:
        SGProblem(8, 2, 2, k, 1e-2, pr.yhat)
    assert abi.STATUS_NAMES[ei.value.status] == "SGOC_ERR_UNSUPPORTED"
    k = pr.kappa.copy()
    k[1, 2, 2] = np.nan
    with pytest.raises(abi.SgocError) as ei:
        SGProblem(8, 2, 2, k, 1e-2, pr.yhat)
    assert abi.STATUS_NAMES[ei.value.status] == "SGOC_ERR_NAN"


def test_device_calls_require_upload():
    sp = _create()
    lib = abi.load()
    st = lib.sgoc_apply_kkt(sp._handle, 0, ctypes.c_void_p(1), ctypes.c_void_p(1), None)
    assert abi.STATUS_NAMES[st] == "SGOC_ERR_NOT_UPLOADED"
    assert "upload" in lib.sgoc_last_error().decode()


def test_hermite_triple_products_match_oracle():
    """The library's Hermite coupling table (the paper's lognormal setting) equals the oracle's
    H_l for every term l >= 1, and the multi-indices are the oracle's."""
    import sg_inputs as si
    from oracle import basis
    from paper_2512_23804_gb300 import SGProblem
    for M, p in [(2, 2), (3, 2), (2, 3)]:
        pr = si.paper_problem(8, M, p)
        sp = SGProblem.from_problem(pr)
        assert np.array_equal(sp.pc_indices(), basis.multi_indices(M, p))
        k, a, b, c = sp.triple_products()
        nA = basis.term_indices(M, p).shape[0]
        H = basis.h_matrices(M, p, nA)
        dense = [np.zeros_like(H[0]) for _ in range(nA)]
        for kk, aa, bb, cc in zip(k, a, b, c):
            dense[kk][aa, bb] = cc
        for l in range(1, nA):
            assert np.max(np.abs(dense[l] - H[l])) <= 1e-15 * max(1.0, np.max(np.abs(H[l]))), l
