"""Launch-shape autotuner (fde_tune_*): the variants of the space-time matvec
(threads per time row) and of the block triangular solves (threads, rows per
register buffer) must give bit-identical results, so tuning can never change a
solution; and a tuned shape is recorded in the table and its cache file."""
import numpy as np
import pytest

import fde_inputs as fi

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    from paper_1305_6653_gb300 import _lib
    lib = _lib.load()
    path = str(tmp_path_factory.mktemp("tune") / "tune.txt")
    lib.fde_tune_cache(path.encode())
    yield lib, path
    for k in (0, 1):
        lib.fde_tune_set(k, -1)
    lib.fde_tune_cache(None)


def _case(m=300):
    # m = 300: several 128-row tiles and a ragged tail; 9 Strang blocks.  m = 500 (m_p = 512):
    # whole 128-wide panels, where the tensor-core LU also writes the strip-major copy of the
    # factor that block-solve shapes 0-2 read (shape 3 reads the row-major planes)
    return fi.manufactured(m, 16, 1.8, "GBDF5", dplus_fn=lambda x: 1 + x, dminus_fn=lambda x: 2 - x)


@pytest.mark.parametrize("precision,m,storage", [("fp64", 300, "fp32"), ("tf32", 300, "fp32"), ("tf32", 500, "fp32"),
                                                 ("bf16", 500, "fp32"), ("tf32", 500, "bf16")])
def test_variants_are_bit_identical(lib, precision, m, storage):
    """With storage "bf16" the register shapes read the bfloat16 copy of the factors; the
    ring shape has no bfloat16 form, so setting 3 launches shape 0 there."""
    from paper_1305_6653_gb300 import FDEProblem, _lib
    L, _ = lib
    prob = _case(m)
    rng = np.random.default_rng(4)
    z = torch.as_tensor(rng.standard_normal(prob.n), device="cuda")
    outs = []
    for v in range(4):  # matvec: 3 shapes (the fourth setting repeats shape 0); block solves: 4
        L.fde_tune_set(_lib.FDE_TUNE_MATVEC, v % 3)
        L.fde_tune_set(_lib.FDE_TUNE_TRSV, v)
        with FDEProblem.from_inputs(prob, device_inputs=True) as p:
            p.assemble().factor(precision, storage=storage)
            y = p.matvec(z).cpu().numpy()
            w = p.precond_apply(z).cpu().numpy()
            x, st = p.solve(tol=1e-11, maxit=400)
            outs.append((y, w, x.cpu().numpy(), st["iterations"]))
    for y, w, x, its in outs[1:]:
        assert np.array_equal(y, outs[0][0])
        assert np.array_equal(w, outs[0][1])
        assert np.array_equal(x, outs[0][2]) and its == outs[0][3]
    for k in (0, 1):
        L.fde_tune_set(k, -1)


def test_autotune_records_the_shape(lib):
    import ctypes as C

    from paper_1305_6653_gb300 import FDEProblem, _lib
    L, path = lib
    prob = fi.manufactured(200, 32, 1.5, "GBDF3")
    mp, nblk = 256, 17
    with FDEProblem.from_inputs(prob) as p:
        p.assemble().factor("fp32")
        x, st = p.solve(tol=1e-10)
    v = C.c_int()
    assert L.fde_tune_query(_lib.FDE_TUNE_MATVEC, mp, prob.s, 0, C.byref(v)) == 0 and 0 <= v.value < 3
    assert L.fde_tune_query(_lib.FDE_TUNE_TRSV, mp, nblk, 1, C.byref(v)) == 0 and 0 <= v.value < 4
    text = open(path).read()
    assert f"matvec 0 {mp} {prob.s} 0 " in text and f"trsv 1 {mp} {nblk} 1 " in text
    # a fresh table read back from the file has the same entries
    L.fde_tune_cache(path.encode())
    assert L.fde_tune_query(_lib.FDE_TUNE_TRSV, mp, nblk, 1, C.byref(v)) == 0 and 0 <= v.value < 4


@pytest.mark.parametrize("precision,m", [("tf32", 700), ("bf16", 700), ("tf32x3", 700), ("tf32", 1000),
                                         ("bf16", 1000), ("tf32x3", 1000)])
def test_lu_interior_variants(lib, precision, m):
    """The interior trailing update of the tensor-core LU as row-pair tiles (variant 0) or
    warp-specialized CTAs with two TMEM accumulators (variant 1): the same MMAs in the same
    K order, so identical factors.  Variant 2 streams C by tensor-map copies and, where
    m_p is a multiple of 128, applies the updates of two consecutive outer steps in one
    pass (one subtraction of the summed products instead of two); elsewhere it is the row
    pairs (identical).  Where it merges, the factors differ from variant 0 by rounding
    only: bounded here by 16 units of the operand precision times the largest factor
    entry.  m = 700: several outer steps, ragged 64-wide tiles; m = 1000: m_p = 1024,
    seven outer steps (three merged pairs and a single step)."""
    from paper_1305_6653_gb300 import FDEProblem, _lib
    L, _ = lib
    prob = fi.manufactured(m, 16, 1.7, "GBDF3", dplus_fn=lambda x: 1 + x, dminus_fn=lambda x: 2 - x)
    facs = []
    for v in (0, 1, 2):
        L.fde_tune_set(_lib.FDE_TUNE_LU, v)
        with FDEProblem.from_inputs(prob) as p:
            p.assemble().factor(precision)
            facs.append([p.factor_block(k) for k in (0, 3, prob.s // 2)])
    L.fde_tune_set(_lib.FDE_TUNE_LU, -1)
    for a, b in zip(facs[0], facs[1]):
        assert np.array_equal(a, b)
    mp = -(-m // 64) * 64
    unit = {"tf32": 2.0 ** -11, "bf16": 2.0 ** -8, "tf32x3": 2.0 ** -22}[precision]
    for a, c in zip(facs[0], facs[2]):
        if mp % 128:
            assert np.array_equal(a, c)
        else:
            d = np.abs(a - c).max() / np.abs(a).max()
            print(precision, m, "merged vs per-step max rel diff", d)
            assert d <= 16 * unit, d
