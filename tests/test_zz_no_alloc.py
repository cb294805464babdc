"""mf_solve_noalloc: the solve entry point for callers that cannot allocate device memory.

Such callers (code that runs inside another runtime's memory pool, plug-ins that must not touch the CUDA
allocator, services that committed all device memory up front) keep the graph and the outputs in device
memory and let the library work in its fixed static scratch area. This test calls the entry point through
the C-ABI twice in a row and checks each result against the regular entry point (mf_solve_device): the
flow value and the minimal source-side cut are unique, so they must match exactly; the per-slot flow must
satisfy the flow definitions. It also checks that the second call leaves the device's free memory as it
was (nothing allocated), and that each kind of bad graph is turned away with its error code before any
solve starts. The file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1507_01926_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def noalloc_fn(mf):
    L = mf.lib()
    f = L.mf_solve_noalloc
    vp = ctypes.c_void_p
    f.argtypes = [ctypes.c_int32, ctypes.c_int32, vp, vp, vp, vp, ctypes.c_int32, ctypes.c_int32, vp, vp, vp, vp]
    f.restype = ctypes.c_int
    return f


def test_no_alloc_matches_regular_entry_point_twice():
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_1507_01926_gb300 import mf

    assert torch.cuda.is_available()
    dev = torch.device("cuda:0")
    fn = noalloc_fn(mf)
    for g in (I.grid2d(70, 90, 17), I.random_graph(3000, 24000, 18, cap=(1, 300))):
        csr = mf.build_csr(g.n, g.tail, g.head, g.cap)
        # regular entry point
        with mf.Graph.from_csr(csr, g.s, g.t) as G:
            ref = G.solve()
        ref_cut = mf.cut_bits_to_bool(ref.cut_bits, g.n)
        # inputs in device memory, int32 layout
        row = torch.from_numpy(csr.row_offsets.astype(np.int32)).to(dev)
        head = torch.from_numpy(csr.head).to(dev)
        cap = torch.from_numpy(csr.cap).to(dev)
        rev = torch.from_numpy(csr.rev.astype(np.int32)).to(dev)
        val = torch.zeros(1, dtype=torch.int64, device=dev)
        flow = torch.zeros(csr.m, dtype=torch.int32, device=dev)
        cutw = torch.zeros((g.n + 31) // 32, dtype=torch.int32, device=dev)
        stream = torch.cuda.current_stream()
        free = []
        for _ in range(2):
            val.fill_(-1)
            flow.fill_(-1)
            cutw.fill_(-1)
            torch.cuda.synchronize()
            rc = fn(g.n, csr.m, row.data_ptr(), head.data_ptr(), cap.data_ptr(), rev.data_ptr(), g.s, g.t,
                    val.data_ptr(), flow.data_ptr(), cutw.data_ptr(), ctypes.c_void_p(stream.cuda_stream))
            assert rc == 0, mf.lib().mf_last_error()
            torch.cuda.synchronize()
            free.append(torch.cuda.mem_get_info()[0])
            assert int(val.item()) == ref.value
            cut = mf.cut_bits_to_bool(cutw.cpu().numpy().view(np.uint32), g.n)
            assert np.array_equal(cut, ref_cut)
            f_in = np.where(csr.arc_slot >= 0, flow.cpu().numpy()[np.maximum(csr.arc_slot, 0)], 0).astype(np.int64)
            assert not oracle.check_flow(g.n, g.s, g.t, g.tail, g.head, g.cap, f_in, ref.value, cut)
        # the first call may load the library's device code (and with it the scratch area); the second
        # call must leave the device's free memory where the first left it
        assert free[1] == free[0], f"free device memory changed by {free[0] - free[1]} bytes across a call"


# Bad graphs in the int32 paired-slot layout (n = 3, s = 0, t = 2) and the code each must give. Every array
# has the length its size argument states, so the input checks themselves stay in bounds.
BAD_GRAPHS = {
    "row offsets not monotone": ([0, 2, 1, 2], [1, 0], [3, 0], [1, 0], -1),
    "head out of range": ([0, 1, 2, 2], [1, 5], [3, 0], [1, 0], -1),
    "rev of a slot is the slot itself": ([0, 1, 2, 2], [1, 0], [3, 0], [0, 0], -1),
    "negative capacity": ([0, 1, 2, 2], [1, 0], [-1, 0], [1, 0], -1),
    "rev[rev[a]] != a": ([0, 2, 3, 4], [1, 2, 0, 0], [3, 4, 0, 0], [2, 2, 0, 1], -2),
    "head[rev[a]] != tail(a)": ([0, 1, 2, 2], [1, 2], [3, 0], [1, 0], -2),
    "pair capacities beyond INT32_MAX": ([0, 1, 2, 2], [1, 0], [2 ** 31 - 1, 1], [1, 0], -4),
}


@pytest.mark.parametrize("case", list(BAD_GRAPHS))
def test_no_alloc_rejects_bad_graphs_before_solving(case):
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_1507_01926_gb300 import mf

    fn = noalloc_fn(mf)
    dev = torch.device("cuda:0")
    row, head, cap, rev, code = BAD_GRAPHS[case]
    m = len(head)
    t32 = lambda a: torch.tensor(a, dtype=torch.int32, device=dev)  # noqa: E731
    row_d, head_d, cap_d, rev_d = t32(row), t32(head), t32(cap), t32(rev)
    val = torch.full((1,), -7, dtype=torch.int64, device=dev)
    flow = torch.full((m,), -7, dtype=torch.int32, device=dev)
    cutw = torch.full((1,), -7, dtype=torch.int32, device=dev)
    rc = fn(3, m, row_d.data_ptr(), head_d.data_ptr(), cap_d.data_ptr(), rev_d.data_ptr(), 0, 2, val.data_ptr(),
            flow.data_ptr(), cutw.data_ptr(), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    assert rc == code, (case, rc, mf.lib().mf_last_error())
    # turned away before the solve: no output was written
    assert int(val.item()) == -7 and (flow == -7).all() and int(cutw.item()) == -7


def test_no_alloc_rejects_graphs_beyond_the_scratch_area():
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_1507_01926_gb300 import mf

    fn = noalloc_fn(mf)
    dev = torch.device("cuda:0")
    n = 1 << 20  # 48 MiB of vertex state alone, beyond the 32 MiB area
    row = torch.zeros(n + 1, dtype=torch.int32, device=dev)
    val = torch.zeros(1, dtype=torch.int64, device=dev)
    rc = fn(n, 0, row.data_ptr(), None, None, None, 0, 1, val.data_ptr(), None, None,
            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == -11
    assert b"scratch" in mf.lib().mf_last_error()
