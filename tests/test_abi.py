"""C ABI of the CUDA library without a GPU: it builds, loads, exports every declared entry
point, and its host-side validation rejects bad problems before touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def gb():
    from paper_2412_17742_gb300 import build
    build.build()
    import paper_2412_17742_gb300 as gb
    gb.load()
    return gb


def declared_functions():
    names = []
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            txt = open(os.path.join(inc, f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"\b(gbsbin_\w+)\s*\(", txt)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(gb):
    names = declared_functions()
    assert len(names) >= 10
    lib = ctypes.CDLL(gb.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
    assert set(gb.EXPORTED) <= set(names)


def test_strerror_and_defaults(gb):
    assert gb.gbsbin_strerror(0) == "ok"
    assert "partition" in gb.gbsbin_strerror(2)
    o = gb.gbsbin_default_options()
    assert (o.precision, o.oversample, o.want_diagnostics, o.tile_override) == (0, 1, 1, 0)


def _status(gb, prob, **opt):
    args = gb.ProblemArgs(prob)
    o = gb.make_options(**opt)
    h = ctypes.c_void_p()
    return gb.load().gbsbin_plan_create(ctypes.byref(args.c), ctypes.byref(o), ctypes.byref(h))


def test_host_validation(gb):
    base = synth.config(0)
    p = synth.config(0)
    p.bin_of_mode = np.array([0, 0, 0, 0], np.int32)
    assert _status(gb, p) == 2                       # empty group
    p = synth.config(0)
    p.bin_of_mode = np.array([0, 1, 2, 1], np.int32)
    assert _status(gb, p) == 2                       # label out of range
    p = synth.config(0)
    p.cutoff = np.array([3, -2], np.int32)
    assert _status(gb, p) == 3
    p = synth.config(0)
    p.cutoff = np.array([9000, 9000], np.int32)
    assert _status(gb, p) == 3                       # grid beyond the limit
    p = synth.config(0)
    p.T = p.T * 2.0
    assert _status(gb, p) == 4                       # amplifying map is not physical
    assert _status(gb, base, oversample=0) == 1
    assert _status(gb, base, precision=7) == 1
    big = synth.random_problem(np.random.default_rng(0), 200, 2, 2, 1)
    assert _status(gb, big) == 8                     # n = 800 > 512
    # nonzero L > M
    p = synth.config(0)
    p.cutoff = np.array([1, 1, 1, 1, 1], np.int32)
    assert _status(gb, p) == 1


def test_nonhermitian_covariance_rejected(gb):
    class Direct:
        pass
    d = Direct()
    d.M, d.K, d.r, d.T = 1, 1, None, None
    d.sigma1 = np.array([[0.5, 0.2], [0.1, 0.5]], complex)
    d.zbar = None
    d.bin_of_mode = np.array([0], np.int32)
    d.cutoff = np.array([4], np.int32)
    assert _status(gb, d) == 4


def test_missing_library_fails_loudly(monkeypatch):
    import paper_2412_17742_gb300 as gb
    monkeypatch.setattr(gb, "_lib", None)
    monkeypatch.setattr(gb, "LIB_PATH", "/nonexistent/libgbsbin.so")
    with pytest.raises(RuntimeError):
        gb.load()


def test_evaluated_digits_cover_half_grid(gb):
    for cut in ([6, 6], [8], [3, 2, 5], [0, 7]):
        dig = gb.evaluated_point_digits(cut)
        radix = [c + 1 for c in cut]
        half = radix[-1] // 2 + 1
        assert len(dig) == int(np.prod(radix[:-1])) * half
        # every grid point is an evaluated point or the conjugate partner of one
        seen = set(map(tuple, dig))
        for k in np.ndindex(*radix):
            neg = tuple((-np.array(k)) % np.array(radix))
            assert k in seen or neg in seen


def _fock_status(gb, prob, **opt):
    args = gb.FockProblemArgs(prob)
    o = gb.make_options(**opt)
    h = ctypes.c_void_p()
    return gb.load().gbsbin_fock_plan_create(ctypes.byref(args.c), ctypes.byref(o), ctypes.byref(h))


def test_fock_host_validation(gb):
    rng = np.random.default_rng(3)

    def fp(**kw):
        p = synth.random_fock_problem(rng, 4, [1, 1, 0, 2], 2, 4)
        for k, v in kw.items():
            setattr(p, k, v)
        return p

    assert _fock_status(gb, fp(bin_of_mode=np.array([0, 0, 0, 0], np.int32))) == 2   # empty group
    assert _fock_status(gb, fp(bin_of_mode=np.array([0, 1, 2, 1], np.int32))) == 2   # label out of range
    assert _fock_status(gb, fp(cutoff=np.array([3, -1], np.int32))) == 3
    assert _fock_status(gb, fp(cutoff=np.array([9000, 9000], np.int32))) == 3         # grid beyond the limit
    assert _fock_status(gb, fp(photons=np.array([1, -1, 0, 0], np.int32))) == 1
    p = fp()
    p.T = p.T * 1.5
    assert _fock_status(gb, p) == 4                                                   # amplifying T
    assert _fock_status(gb, fp(), want_backward=True) == 8
    assert _fock_status(gb, fp(), shard=(0, 99)) == 1                                 # beyond the nodes
    assert _fock_status(gb, fp(), tile_override=5) == 1
    assert _fock_status(gb, fp(), oversample=0) == 1
    big = synth.random_fock_problem(rng, 40, [1] * 33 + [0] * 7, 2, 2)
    assert _fock_status(gb, big) == 8                                                 # 33 occupied inputs
    many = synth.random_fock_problem(rng, 9, [1] * 9, 9, 1)
    assert _fock_status(gb, many) == 8                                                # 9 groups > 8
    nodes = synth.random_fock_problem(rng, 31, [3] * 31, 1, 4)
    assert _fock_status(gb, nodes) == 8                                               # 4^30 nodes


@pytest.mark.parametrize("tree", [11, 12], ids=["df32", "fp64"])
def test_tree_kernel_validation(gb, tree):
    one_group = synth.random_problem(np.random.default_rng(7), 4, 1, 1, 3)
    assert _status(gb, one_group, tile_override=tree) == 8               # the tree needs L >= 2
    big = synth.random_problem(np.random.default_rng(8), 40, 1, 2, 2)    # n = 80 > 64
    assert _status(gb, big, tile_override=tree) == 8
    assert _status(gb, synth.config(1), tile_override=tree, shard=(0, 10)) == 8
    assert _status(gb, synth.config(1), tile_override=9) == 1            # a Fock kernel id
    assert _status(gb, synth.config(1), tile_override=15) == 1           # no such kernel


@pytest.mark.parametrize("btree", [13, 14], ids=["df32", "fp64"])
def test_large_tree_validation(gb, btree):
    # the large-matrix tree's host-side refusals (before any device call)
    one_group = synth.random_problem(np.random.default_rng(7), 4, 1, 1, 3)
    assert _status(gb, one_group, tile_override=btree) == 8              # needs L >= 2
    big_last = synth.random_problem(np.random.default_rng(9), 100, 1, 2, 2)   # last group 194 rows > 192
    big_last.bin_of_mode = np.array([0] * 3 + [1] * 97, np.int32)
    assert _status(gb, big_last, tile_override=btree) == 8


def _herald_status(gb, state, roles, cutoff, cut, **opt):
    args = gb.HeraldProblemArgs(state, roles, cutoff, cut)
    o = gb.make_options(**opt)
    h = ctypes.c_void_p()
    return gb.load().gbsbin_herald_plan_create(ctypes.byref(args.c), ctypes.byref(o), ctypes.byref(h))


def test_herald_host_validation(gb):
    rng = np.random.default_rng(805)
    st = synth.random_problem(rng, 4, 1, 2, [2, 2], displaced=True)
    ok = ([0, 1, -2, -1], [2, 2], 3)
    assert _herald_status(gb, st, [0, 1, -2, 2], [2, 2], 3) == 1          # role outside [-2, L)
    assert _herald_status(gb, st, [0, 1, -3, -1], [2, 2], 3) == 1
    assert _herald_status(gb, st, [0, 0, -2, -1], [2, 2], 3) == 2         # group 1 has no mode
    assert _herald_status(gb, st, [0, 1, -1, -1], [2, 2], 3) == 8         # nothing kept
    assert _herald_status(gb, st, *ok[:2], -1) == 1                      # fock cutoff < 0
    assert _herald_status(gb, st, [0, 1, -2, -1], [2, -1], 3) == 3        # heralding cutoff < 0
    assert _herald_status(gb, st, *ok, precision=1) == 1                  # FP64 only
    assert _herald_status(gb, st, *ok, want_backward=True) == 1
    assert _herald_status(gb, st, *ok, shard=(0, 4)) == 1
    assert _herald_status(gb, st, *ok, tile_override=3) == 1
    big = synth.random_problem(rng, 25, 2, 1, [2])                         # 2 M K = 100 > 96
    assert _herald_status(gb, big, [0] * 48 + [-2, -2], [2], 2) == 8
    five = synth.random_problem(rng, 6, 1, 1, [2])
    assert _herald_status(gb, five, [0, -2, -2, -2, -2, -2], [2], 1) == 8   # five kept modes
    assert _herald_status(gb, five, [0, 0, -2, -2, -2, -1], [2], 10) == 8   # 11^6 coefficients
    bad = synth.random_problem(rng, 4, 1, 2, [2, 2])
    bad.T = 1.5 * np.eye(4)                                                # ||T|| > 1
    assert _herald_status(gb, bad, *ok) == 4
