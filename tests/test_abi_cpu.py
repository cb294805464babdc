"""CPU checks of the C-ABI library: it loads, exports every entry point include/mf.h declares, the
host-side CSR builder pairs reverse slots correctly, and argument errors are reported without a GPU."""
import os
import re

import numpy as np
import pytest

from paper_1507_01926_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "mf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mf_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol(built):
    import ctypes

    from paper_1507_01926_gb300 import mf

    L = ctypes.CDLL(mf.LIB_PATH)
    names = declared_functions()
    assert "mf_solve" in names and "mf_create_graph" in names
    missing = [nm for nm in names if not hasattr(L, nm)]
    assert not missing, f"declared but not exported: {missing}"


def test_default_options(built):
    from paper_1507_01926_gb300 import mf

    o = mf.default_options()
    assert o.gr_freq == 0.5 and o.gr_alpha == 6 and o.work_beta == 12
    assert o.block_threads % 32 == 0 and o.timeout_ms > 0
    so = mf.service_default_options()
    assert so.block_threads == 128
    assert all(getattr(so, k) == getattr(o, k) for k, _ in mf.Options._fields_ if k != "block_threads")


def check_csr(c, tail, head, cap):
    from paper_1507_01926_gb300 import mf  # noqa: F401

    m = c.m
    r = c.rev
    assert (r[r] == np.arange(m)).all(), "rev is not an involution"
    assert (r != np.arange(m)).all()
    t = c.tails()
    assert (c.head[r] == t).all(), "head[rev[a]] != tail(a)"
    assert np.all(np.diff(c.row_offsets) >= 0) and c.row_offsets[0] == 0 and c.row_offsets[-1] == m
    keep = tail != head
    a = c.arc_slot
    assert (a[~keep] == -1).all()
    assert (t[a[keep]] == tail[keep]).all() and (c.head[a[keep]] == head[keep]).all()
    assert (c.cap[a[keep]] == cap[keep]).all()
    # every slot holds at most one input arc; slots without one have capacity 0
    owned = np.zeros(m, bool)
    owned[a[keep]] = True
    assert owned.sum() == keep.sum()
    assert (c.cap[~owned] == 0).all()
    # rows sorted by head
    for v in range(c.n):
        h = c.head[c.row_offsets[v]:c.row_offsets[v + 1]]
        assert (np.diff(h) >= 0).all()


@pytest.mark.parametrize("seed", range(12))
def test_build_csr_random_multigraph(built, seed):
    from paper_1507_01926_gb300 import mf

    g = I.random_graph(int(5 + seed * 3), 40 + 10 * seed, seed, cap=(0, 50), allow_loops=True)
    c = mf.build_csr(g.n, g.tail, g.head, g.cap)
    check_csr(c, g.tail, g.head, g.cap)
    assert c.dropped_self_loops == int((g.tail == g.head).sum())


def test_build_csr_pairs_antiparallel_arcs(built):
    from paper_1507_01926_gb300 import mf

    tail = np.array([0, 1, 0, 1, 2, 0], np.int32)
    head = np.array([1, 0, 1, 2, 1, 1], np.int32)
    cap = np.array([5, 7, 3, 4, 6, 9], np.int32)
    c = mf.build_csr(3, tail, head, cap)
    check_csr(c, tail, head, cap)
    # 0->1 (arcs 0,2,5) against 1->0 (arc 1): arc 0 pairs with arc 1; 1->2 pairs with 2->1
    a = c.arc_slot
    assert c.rev[a[0]] == a[1]
    assert c.rev[a[3]] == a[4]
    assert c.m == 2 * 4  # pairs: (0,1), (2,-), (3,4), (5,-)


def test_build_csr_grid_slot_count(built):
    from paper_1507_01926_gb300 import mf

    g = I.grid2d_64x64()
    c = mf.build_csr(g.n, g.tail, g.head, g.cap)
    assert c.m == 24320
    check_csr(c, g.tail, g.head, g.cap)


def test_build_csr_rejects_bad_input(built):
    from paper_1507_01926_gb300 import mf

    with pytest.raises(mf.MFError) as e:
        mf.build_csr(3, [0], [3], [1])
    assert e.value.code == -1
    with pytest.raises(mf.MFError) as e:
        mf.build_csr(3, [0], [1], [-1])
    assert e.value.code == -1
    with pytest.raises(mf.MFError) as e:
        mf.build_csr(3, [0, 1], [1, 0], [2 ** 31 - 1, 1])
    assert e.value.code == -4
    c = mf.build_csr(3, [0, 1], [1, 0], [2 ** 31 - 2, 1])
    assert c.m == 2


def test_create_graph_argument_errors_without_gpu(built):
    from paper_1507_01926_gb300 import mf

    z32, z64 = np.zeros(0, np.int32), np.zeros(0, np.int64)
    with pytest.raises(mf.MFError) as e:
        mf.Graph(3, np.zeros(4, np.int64), z32, z32, z64, 1, 1)
    assert e.value.code == -3
    with pytest.raises(mf.MFError) as e:
        mf.Graph(1, np.zeros(2, np.int64), z32, z32, z64, 0, 0)
    assert e.value.code == -1
    with pytest.raises(mf.MFError) as e:
        mf.Graph(3, np.zeros(4, np.int64), z32, z32, z64, 0, 5)
    assert e.value.code == -1
    with pytest.raises(mf.MFError) as e:
        mf.Graph(3, np.zeros(4, np.int64), z32, z32, z64, 0, 2, mf.default_options(block_threads=100))
    assert e.value.code == -1


@pytest.mark.parametrize("field,bad", [("use_graph", 2), ("local_lists", -1), ("local_lists", 16), ("local_lists", 1024),
                                       ("bfs_hops", 0), ("bfs_hops", 65), ("bin_thread", 16), ("bin_thread", 17),
                                       ("kernel_variant", 5), ("gap_every", -1), ("bfs_pull", -1),
                                       ("union_max_requests", -1)])
def test_out_of_range_options_rejected_without_gpu(built, field, bad):
    from paper_1507_01926_gb300 import mf

    o = mf.default_options()
    assert (o.use_graph, o.local_lists, o.bfs_hops, o.gap_every, o.bfs_pull) == (0, 1, 8, 0, 50)
    z32, z64 = np.zeros(0, np.int32), np.zeros(0, np.int64)
    with pytest.raises(mf.MFError) as e:
        mf.Graph(3, np.zeros(4, np.int64), z32, z32, z64, 0, 2, mf.default_options(**{field: bad}))
    assert e.value.code == -1 and field in str(e.value)


def test_struct_sizes_match_the_binding(built):
    import ctypes

    from paper_1507_01926_gb300 import mf

    L = mf.lib()  # also checks the sizes when it loads
    ob, sb = ctypes.c_int32(), ctypes.c_int32()
    L.mf_struct_sizes(ctypes.byref(ob), ctypes.byref(sb))
    assert (ob.value, sb.value) == (ctypes.sizeof(mf.Options), ctypes.sizeof(mf.Stats))
    L.mf_struct_sizes(None, None)  # both nullable


def _struct_fields(src, name):
    """Field names, in order, of `typedef struct name { ... } name;` in the header (comments removed)."""
    import re

    body = re.search(r"typedef struct %s \{(.*?)\} %s;" % (name, name), src, re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    names = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        decl = re.sub(r"\[\d+\]", "", decl)  # arrays: the name is what matters
        typ, rest = decl.split(None, 1) if " " in decl else (decl, "")
        names += [x.strip().lstrip("*") for x in rest.split(",")]
    return names


def test_binding_structs_follow_the_header(built):
    """mf.py's ctypes copies of mf_options and mf_stats have the header's fields in the header's order."""
    from paper_1507_01926_gb300 import mf

    src = open(os.path.join(ROOT, "include", "mf.h")).read()
    assert _struct_fields(src, "mf_options") == [f for f, _ in mf.Options._fields_]
    assert _struct_fields(src, "mf_stats") == [f for f, _ in mf.Stats._fields_]
