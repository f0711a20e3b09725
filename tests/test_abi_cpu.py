"""C-ABI checks that need no GPU: the library loads, exports every entry point the
header declares, validates descriptors, and its host planner produces exactly the
oracle's level structure (greedy colours, merged near/fill block CSR and kinds)."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import structure as st

from conftest import ROOT, problem

HEADER = os.path.join(ROOT, "include", "h2rs.h")


def _declared():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"H2_API\s+[\w\s\*]+?\b(h2_\w+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    from paper_2509_11152_b300 import binding
    lib = binding.lib()
    names = _declared()
    assert len(names) >= 12
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(binding.EXPORTED) == names
    assert binding.h2_version().startswith("h2rs")


def _oracle_levels(A):
    """Oracle structure of every skeletonised level (leaves first)."""
    t = A.top_level()
    out = []
    carried = set()
    for l in range(A.depth, t - 1, -1):
        nbrs = st.neighbours(A, l)
        fill = st.fill_pattern(nbrs, carried)
        lay = st.level_layout(nbrs, fill, [1] * len(nbrs))
        out.append((st.greedy_colouring(nbrs), lay))
        pn = st.neighbours(A, l - 1)
        pnear = {(p, q) for p in range(len(pn)) for q in pn[p]}
        carried = st.carried_to_parent(fill, pnear)
    return out


@pytest.mark.parametrize("name,over", [
    ("cov2d", dict(n=1024, leaf=32)),
    ("cov2d", {}),
    ("laplace2d", dict(n=4096, leaf=32, eta=0.7)),
    ("matern3d", dict(n=2048, leaf=32)),
    ("sphere", dict(n=8192, leaf=64)),
    ("gauss3d", dict(n=1500, leaf=32)),
    ("helmholtz3d", dict(n=4096, leaf=64)),
    ("lru3d", dict(n=4096, leaf=64)),
])
def test_plan_matches_oracle_structure(name, over):
    from paper_2509_11152_b300 import h2_plan_query
    A = problem(name, **over).A
    for li, (colour, lay) in enumerate(_oracle_levels(A)):
        q = h2_plan_query(A, li)
        assert np.array_equal(q["colour"], np.asarray(colour, np.int32))
        assert np.array_equal(q["row_ptr"], lay["row_ptr"])
        assert np.array_equal(q["col"], lay["col"])
        assert np.array_equal(q["kind"], lay["kind"].astype(np.int32))


def test_descriptor_validation_errors():
    from paper_2509_11152_b300 import binding
    A = problem("cov2d", n=512, leaf=32).A
    d, keep = binding.make_desc(A)
    nbox = ctypes.c_int64()
    rc = binding.lib().h2_plan_query(ctypes.byref(d), 0, ctypes.byref(nbox), None, None, None, None, None)
    assert rc == 0 and nbox.value == 16
    # a child range that does not partition its parent
    bad = keep["node_size"].copy()
    bad[1] += 1
    d.node_size = bad.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    rc = binding.lib().h2_plan_query(ctypes.byref(d), 0, None, None, None, None, None, None)
    assert rc == -1 and b"partition" in binding.lib().h2_last_error()
    d.node_size = keep["node_size"].ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    # an inadmissible pattern that is not symmetric: one leaf entry (g, t) moved to
    # (g, t+1), keeping the row sorted and every block size (all leaves hold 32 points)
    ptr, col = keep["inad_ptr"], keep["inad_col"].copy()
    first_leaf = (1 << A.depth) - 1
    e = next(e for g in range(first_leaf, len(ptr) - 1) for e in range(ptr[g], ptr[g + 1] - 1)
             if col[e] != g and col[e] + 1 < col[e + 1] and col[e] + 1 != g)
    col[e] += 1
    d.inad_col = col.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    rc = binding.lib().h2_plan_query(ctypes.byref(d), 0, None, None, None, None, None, None)
    assert rc == -1 and b"not symmetric" in binding.lib().h2_last_error()
    d.inad_col = keep["inad_col"].ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    # an admissible pattern that is not symmetric: the entry (t, g) of one admissible
    # pair removed (with its coupling's slot), (g, t) kept
    aptr, acol, soff = keep["adm_ptr"], keep["adm_col"], keep["S_off"]
    g = next(g for g in range(len(aptr) - 1) if aptr[g + 1] > aptr[g])
    t = acol[aptr[g]]
    e2 = aptr[t] + int(np.searchsorted(acol[aptr[t]:aptr[t + 1]], g))
    assert acol[e2] == g
    aptr2 = aptr.copy()
    aptr2[t + 1:] -= 1
    acol2 = np.delete(acol, e2)
    soff2 = np.concatenate([soff[:e2 + 1], soff[e2 + 2:] - (soff[e2 + 1] - soff[e2])])
    d.adm_ptr = aptr2.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    d.adm_col = acol2.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    d.S_off = soff2.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    rc = binding.lib().h2_plan_query(ctypes.byref(d), 0, None, None, None, None, None, None)
    assert rc == -1 and b"admissible pattern is not symmetric" in binding.lib().h2_last_error()
    d.adm_ptr = aptr.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    d.adm_col = acol.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    d.S_off = soff.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    rc = binding.lib().h2_plan_query(ctypes.byref(d), 0, None, None, None, None, None, None)
    assert rc == 0
    # a level out of range
    rc = binding.lib().h2_plan_query(ctypes.byref(d), 99, None, None, None, None, None, None)
    assert rc == -1
    # a null descriptor
    rc = binding.lib().h2_plan_query(None, 0, None, None, None, None, None, None)
    assert rc == -1


def _small_batch():
    from h2gen import make_batch
    from conftest import problem as pr
    batch = make_batch("gauss3d", nsys=4, nmin=300, nmax=3000, leaf=32)
    # plus one system with no admissible block (its top matrix is its leaf near field)
    return [pb.A for pb in batch] + [pr("cov2d", n=256, leaf=16, eta=1e-6).A]


def test_uneven_sizes_are_log_uniform_and_seeded():
    from h2gen import uneven_sizes
    n = uneven_sizes()
    assert n == uneven_sizes() and len(n) == 64
    assert min(n) >= 2048 and max(n) <= 131072
    # log-uniform: about half the systems below the geometric mean sqrt(2048 * 131072)
    assert 20 <= sum(v < 16384 for v in n) <= 44


def test_batch_plan_is_the_union_of_the_single_plans():
    """Forest levels aligned by height: every system's boxes, colours and block rows at
    forest level a equal its own plan at level a (shifted by its box offset); its top
    boxes sit at the level after its last skeletonised one; boxes above are inert."""
    from paper_2509_11152_b300 import h2_plan_query, h2_plan_query_batch
    As = _small_batch()
    depths = [A.depth for A in As]
    assert len(set(depths)) >= 3                    # genuinely uneven
    nlev = [0 if A.top_level() is None else A.depth - A.top_level() + 1 for A in As]
    for a in range(max(nlev) + 1):
        q = h2_plan_query_batch(As, a)
        for z, A in enumerate(As):
            boxes = np.flatnonzero(q["system"] == z)
            assert len(boxes) == 1 << (A.depth - a) if a <= A.depth else len(boxes) == 0
            if not len(boxes):
                continue
            assert np.array_equal(boxes, np.arange(boxes[0], boxes[0] + len(boxes)))
            st_ = q["state"][boxes]
            rows = [q["col"][q["row_ptr"][i]:q["row_ptr"][i + 1]] - boxes[0] for i in boxes]
            kinds = [q["kind"][q["row_ptr"][i]:q["row_ptr"][i + 1]] for i in boxes]
            if a < nlev[z]:
                assert (st_ == 1).all()
                s1 = h2_plan_query(A, a)
                assert np.array_equal(q["colour"][boxes], s1["colour"])
                for i, (r, k) in enumerate(zip(rows, kinds)):
                    lo, hi = s1["row_ptr"][i], s1["row_ptr"][i + 1]
                    assert np.array_equal(r, s1["col"][lo:hi]) and np.array_equal(k, s1["kind"][lo:hi])
            elif a == nlev[z]:
                assert (st_ == 2).all() and (q["colour"][boxes] == -1).all()
                for r, k in zip(rows, kinds):          # dense top matrix: all pairs near
                    assert np.array_equal(r, np.arange(len(boxes))) and (k == 0).all()
            else:
                assert (st_ == 0).all() and all(len(r) == 0 for r in rows)


def test_batch_plan_edge_cases():
    """A batch mixing a single-box system (depth 0), a system with nothing admissible
    and a regular one: the lone box and the dense system are top boxes at the leaf
    level, and a batch of one equals the single plan."""
    from paper_2509_11152_b300 import h2_plan_query, h2_plan_query_batch
    from paper_2509_11152_b300 import binding
    lone = problem("cov2d", n=50, leaf=64).A
    dense_sys = problem("cov2d", n=256, leaf=16, eta=1e-6).A
    reg = problem("cov2d", n=1024, leaf=32).A
    q = h2_plan_query_batch([lone, dense_sys, reg], 0)
    for z, A in enumerate([lone, dense_sys]):
        boxes = np.flatnonzero(q["system"] == z)
        assert len(boxes) == 1 << A.depth and (q["state"][boxes] == 2).all()
    assert (q["state"][q["system"] == 2] == 1).all()
    one = h2_plan_query_batch([reg], 0)
    single = h2_plan_query(reg, 0)
    for key in ("colour", "row_ptr", "col", "kind"):
        assert np.array_equal(one[key], single[key])
    # bad arguments are reported, not trapped
    d, keep = binding.make_desc(reg)
    arr = (binding.h2_matrix_desc * 1)(d)
    assert binding.lib().h2_plan_query_batch(0, arr, 0, None, None, None, None, None, None, None, None) == -1
    assert binding.lib().h2_plan_query_batch(1, None, 0, None, None, None, None, None, None, None, None) == -1
    assert binding.lib().h2_plan_query_batch(1, arr, 99, None, None, None, None, None, None, None, None) == -1


def test_empty_and_oversized_descriptors_are_rejected():
    """n = 0 and absurd depths are argument errors (reported, not trapped)."""
    from paper_2509_11152_b300 import binding
    A = problem("cov2d", n=512, leaf=32).A
    d, keep = binding.make_desc(A)
    lib = binding.lib()
    for field, bad in (("n", 0), ("n", -5), ("depth", -1), ("depth", 40)):
        old = getattr(d, field)
        setattr(d, field, bad)
        rc = lib.h2_plan_query(ctypes.byref(d), 0, None, None, None, None, None, None)
        assert rc == -1, (field, bad)
        setattr(d, field, old)
    assert lib.h2_plan_query(ctypes.byref(d), 0, None, None, None, None, None, None) == 0


def test_plain_c_caller_builds_and_plans():
    """The C-ABI is usable from plain C (no torch, no Python): the example builds with
    gcc against include/h2rs.h and libh2rs.so and runs the host-only plan query."""
    import shutil
    import subprocess
    import tempfile
    from paper_2509_11152_b300 import binding
    binding.lib()                                     # the library is built
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = os.path.join(ROOT, "paper_2509_11152_b300", "examples", "plan_query.c")
    libdir = os.path.dirname(binding.LIB_PATH)
    with tempfile.TemporaryDirectory() as td:
        exe = os.path.join(td, "plan_query")
        r = subprocess.run([cc, "-std=c99", "-Wall", "-Werror", src, "-I", os.path.join(ROOT, "include"),
                            "-L", libdir, "-lh2rs", f"-Wl,-rpath,{libdir}", "-o", exe],
                           capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
        r = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, r.stdout + r.stderr
    lines = r.stdout.splitlines()
    assert lines[0].startswith("h2rs")
    assert "4 boxes, 14 blocks" in lines[1]
    assert lines[2] == "box 0 colour 0: 0 1 2f"          # distance-two fill through box 1
    assert "partition" in lines[-1]


def test_binding_rejects_malformed_vectors():
    """The binding only marshals: non-float64 or row-major right-hand sides are refused
    before anything reaches the library (no GPU needed)."""
    import torch
    from paper_2509_11152_b300 import binding
    with pytest.raises(TypeError):
        binding._vec(torch.zeros(8, dtype=torch.float32))
    with pytest.raises(ValueError):
        binding._vec(torch.zeros(8, 3, dtype=torch.float64))           # row-major (n, nrhs)
    p, nrhs, ld, dev = binding._vec(binding.colmajor(torch.zeros(8, 3, dtype=torch.float64)))
    assert nrhs == 3 and ld == 8 and dev == 0
    p, nrhs, ld, dev = binding._vec(torch.zeros(8, dtype=torch.float64))
    assert nrhs == 1 and ld == 8


def test_every_declared_entry_point_is_documented():
    """Each entry point of the header carries a comment block that states its errors or
    its return value (the boundary's documentation contract)."""
    txt = open(HEADER).read()
    for name in _declared():
        i = txt.index(name + "(")
        before = txt[max(0, i - 1500):i]
        assert "/*" in before, name


def _structure_only(pts, leaf, eta):
    """An H^2 descriptor's index arrays from a point set (tree + partition only; rank 1
    everywhere, values never read by the host planner) and an object the oracle's
    structure functions accept."""
    import types
    import torch
    from h2gen.tree import build_kdtree, dual_traversal
    tree = build_kdtree(pts, leaf)
    part = dual_traversal(tree, eta)
    d = tree.depth
    nn = (1 << (d + 1)) - 1
    rank = np.ones(nn, np.int64)
    leaves = np.arange((1 << d) - 1, nn)
    U_off = np.concatenate([[0], np.cumsum(tree.size[leaves])]).astype(np.int64)
    E_off = np.concatenate([[0, 0], np.arange(1, nn)]).astype(np.int64)
    adm = np.concatenate([part.adm[l] for l in range(d + 1)], axis=0)
    inad = np.concatenate([part.inad[l] for l in range(d + 1)], axis=0)
    S = types.SimpleNamespace(
        n=int(tree.size[0]), depth=d, node_start=tree.start, node_size=tree.size, rank=rank, U_off=U_off,
        E_off=E_off, adm_ptr=np.concatenate([[0], np.cumsum(np.bincount(adm[:, 0], minlength=nn))]),
        adm_col=adm[:, 1], S_off=np.arange(len(adm) + 1),
        inad_ptr=np.concatenate([[0], np.cumsum(np.bincount(inad[:, 0], minlength=nn))]), inad_col=inad[:, 1],
        D_off=np.concatenate([[0], np.cumsum(tree.size[part.inad[d][:, 0]] * tree.size[part.inad[d][:, 1]])]),
        U=torch.zeros(1, dtype=torch.float64), E=torch.zeros(1, dtype=torch.float64),
        S=torch.zeros(1, dtype=torch.float64), D=torch.zeros(1, dtype=torch.float64))

    def top_level():
        for l in range(d + 1):
            f, c = (1 << l) - 1, 1 << l
            if S.adm_ptr[f + c] - S.adm_ptr[f] > 0:
                return l
        return None
    S.top_level = top_level
    return S


@pytest.mark.parametrize("seed", range(16))
def test_plan_matches_oracle_on_random_structures(seed):
    """Random point sets (2D / 3D, uniform or clustered), leaf sizes and admissibility
    parameters: the library's host plan equals the oracle's level structure bit for
    bit at every skeletonised level."""
    import ctypes
    from paper_2509_11152_b300 import binding
    rng = np.random.default_rng(1000 + seed)
    dim = int(rng.integers(2, 4))
    n = int(rng.integers(200, 3000))
    pts = rng.random((n, dim))
    if seed % 2:                                       # clustered: uneven box geometry
        pts = np.concatenate([pts[: n // 2] * 0.2, pts[n // 2:]])
    leaf = int(rng.choice([8, 16, 32, 64]))
    eta = float(rng.choice([0.5, 0.7, 1.0, 2.0]))
    A = _structure_only(pts, leaf, eta)
    desc = binding.h2_matrix_desc()
    desc.n = A.n
    desc.depth = A.depth
    keep = {}
    for name in ("node_start", "node_size", "rank", "U_off", "E_off", "adm_ptr", "adm_col", "S_off",
                 "inad_ptr", "inad_col", "D_off"):
        arr = np.ascontiguousarray(np.asarray(getattr(A, name), np.int64))
        keep[name] = arr
        setattr(desc, name, arr.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
    for name in ("U", "E", "S", "D"):
        setattr(desc, name, ctypes.cast(ctypes.c_void_p(A.U.data_ptr()), ctypes.POINTER(ctypes.c_double)))
    lib = binding.lib()
    levels = _oracle_levels(A) if A.top_level() is not None else []
    assert len(levels) >= 1 or A.top_level() is None
    for li, (colour, lay) in enumerate(levels):
        nbox, nblk = ctypes.c_int64(), ctypes.c_int64()
        assert lib.h2_plan_query(ctypes.byref(desc), li, ctypes.byref(nbox), ctypes.byref(nblk),
                                 None, None, None, None) == 0, binding.lib().h2_last_error()
        col_ = np.zeros(nbox.value, np.int32)
        rp = np.zeros(nbox.value + 1, np.int64)
        cl = np.zeros(nblk.value, np.int64)
        kd = np.zeros(nblk.value, np.int32)
        lib.h2_plan_query(ctypes.byref(desc), li, None, None, binding._ptr(col_, ctypes.c_int32),
                          binding._ptr(rp, ctypes.c_int64), binding._ptr(cl, ctypes.c_int64),
                          binding._ptr(kd, ctypes.c_int32))
        assert np.array_equal(col_, np.asarray(colour, np.int32))
        assert np.array_equal(rp, lay["row_ptr"]) and np.array_equal(cl, lay["col"])
        assert np.array_equal(kd, lay["kind"].astype(np.int32))


def test_batch_plan_on_random_forests():
    """Random batches of random structures (different depths and tops): at every forest
    level each system's boxes, colours, rows and states equal its own plan."""
    from paper_2509_11152_b300 import h2_plan_query, h2_plan_query_batch
    rng = np.random.default_rng(77)
    for trial in range(3):
        As = []
        for z in range(int(rng.integers(2, 6))):
            dim = int(rng.integers(2, 4))
            pts = rng.random((int(rng.integers(100, 2500)), dim))
            As.append(_structure_only(pts, int(rng.choice([16, 32])), float(rng.choice([0.7, 1.0]))))
        nlev = [0 if A.top_level() is None else A.depth - A.top_level() + 1 for A in As]
        for a in range(max(nlev) + 1):
            q = h2_plan_query_batch(As, a)
            for z, A in enumerate(As):
                boxes = np.flatnonzero(q["system"] == z)
                if a > A.depth:
                    assert len(boxes) == 0
                    continue
                assert np.array_equal(boxes, np.arange(boxes[0], boxes[0] + len(boxes)))
                if a < nlev[z]:
                    s1 = h2_plan_query(A, a)
                    assert (q["state"][boxes] == 1).all()
                    assert np.array_equal(q["colour"][boxes], s1["colour"])
                    for i, bi in enumerate(boxes):
                        r = q["col"][q["row_ptr"][bi]:q["row_ptr"][bi + 1]] - boxes[0]
                        assert np.array_equal(r, s1["col"][s1["row_ptr"][i]:s1["row_ptr"][i + 1]])
                else:
                    assert (q["state"][boxes] == (2 if a == nlev[z] else 0)).all()


def test_missing_library_fails_loudly():
    """No fallback: without the built library every entry point raises."""
    import subprocess
    import sys
    code = ("from paper_2509_11152_b300 import binding\n"
            "binding.LIB_PATH = '/nonexistent/libh2rs.so'\n"
            "binding._lib = None\n"
            "try:\n"
            "    binding.lib()\n"
            "except RuntimeError as e:\n"
            "    print('RAISED', e)\n")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and "RAISED" in r.stdout and "missing" in r.stdout, r.stdout + r.stderr


def test_product_code_never_touches_the_oracle():
    """The library package and the input generators import nothing from oracle/."""
    import re
    for pkg in ("paper_2509_11152_b300", "h2gen"):
        for dirpath, _, files in os.walk(os.path.join(ROOT, pkg)):
            for f in files:
                if f.endswith((".py", ".cu", ".cuh", ".cpp", ".h", ".c")):
                    src = open(os.path.join(dirpath, f)).read()
                    assert not re.search(r"^\s*(from|import)\s+oracle\b|#include\s+\S*oracle", src, re.M), f


def _example_matrix():
    """The H^2 matrix that examples/solve.c builds, mirrored here (same arrays)."""
    import math
    import torch
    from h2gen.h2matrix import H2Matrix

    def kern(i, j):
        xi, xj = (i + 0.5) / 8, (j + 0.5) / 8
        return 1.1 if i == j else math.exp(-abs(xi - xj) / 0.5)
    start = np.array([0, 0, 4, 0, 2, 4, 6])
    adm_ptr = np.array([0, 0, 0, 0, 2, 3, 4, 6])
    adm_col = np.array([5, 6, 6, 3, 3, 4])
    inad_ptr = np.array([0, 1, 3, 5, 7, 10, 13, 15])
    inad_col = np.array([0, 1, 2, 1, 2, 3, 4, 3, 4, 5, 4, 5, 6, 5, 6])
    S = [0.5 * sum(kern(start[s] + a, start[t] + b) for a in range(2) for b in range(2))
         for s in range(3, 7) for t in adm_col[adm_ptr[s]:adm_ptr[s + 1]]]
    D = [kern(start[s] + r, start[t] + c) for s in range(3, 7) for t in inad_col[inad_ptr[s]:inad_ptr[s + 1]]
         for c in range(2) for r in range(2)]
    f = lambda v: torch.tensor(v, dtype=torch.float64)
    return H2Matrix(n=8, depth=2, node_start=start, node_size=np.array([8, 4, 4, 2, 2, 2, 2]),
                    rank=np.ones(7, np.int64), U_off=np.array([0, 2, 4, 6, 8]), U=f([2 ** -0.5] * 8),
                    E_off=np.array([0, 0, 1, 2, 3, 4, 5, 6]), E=f([2 ** -0.5] * 6), adm_ptr=adm_ptr,
                    adm_col=adm_col, S_off=np.arange(7), S=f(S), inad_ptr=inad_ptr, inad_col=inad_col,
                    D_off=np.arange(0, 44, 4), D=f(D))


def test_c_solve_example_matrix_and_build():
    """examples/solve.c: its matrix is a valid symmetric positive definite H^2 matrix
    that the oracle factorises to the dense solution; the program builds with gcc
    (-Wall -Werror) and, run without a GPU, ends with a status code, not a crash (on
    a GPU it prints two backward errors and exits 0)."""
    import shutil
    import subprocess
    import tempfile
    import torch
    from oracle import dense, rs
    from paper_2509_11152_b300 import binding
    A = _example_matrix().numpy()
    M = dense.expand(A)
    assert np.allclose(M, M.T) and np.linalg.eigvalsh(M).min() > 0.05
    b = np.ones((8, 1))
    norm_a = np.linalg.norm(M, 2)
    Z = rs.factorize(A, 1e-12, norm_a)
    assert np.allclose(rs.solve(Z, b), np.linalg.solve(M, b), rtol=1e-12)
    binding.lib()
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = os.path.join(ROOT, "paper_2509_11152_b300", "examples", "solve.c")
    libdir = os.path.dirname(binding.LIB_PATH)
    with tempfile.TemporaryDirectory() as td:
        exe = os.path.join(td, "solve")
        r = subprocess.run([cc, "-std=c99", "-Wall", "-Werror", src, "-I", os.path.join(ROOT, "include"),
                            "-L", libdir, "-lh2rs", "-lm", f"-Wl,-rpath,{libdir}", "-o", exe],
                           capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
        r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    if torch.cuda.is_available():
        assert r.returncode == 0, r.stdout + r.stderr
        assert "float64 factor + solve" in r.stdout and "float32 factor" in r.stdout
    else:
        assert r.returncode == 2 and "h2_matrix_create failed" in r.stderr, r.stdout + r.stderr
