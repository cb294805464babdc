"""mf_solve_noalloc: the solve entry point for callers that cannot allocate device memory.

Such callers (code that runs inside another runtime's memory pool, plug-ins that must not touch the CUDA
allocator, services that committed all device memory up front) keep the graph and the outputs in device
memory and let the library work in its fixed static scratch area. This test calls the entry point through
the C-ABI twice in a row and checks each result against the regular entry point (mf_solve_device): the
flow value and the minimal source-side cut are unique, so they must match exactly; the per-slot flow must
satisfy the flow definitions. The file is named so that pytest collects it last.
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
        for _ in range(2):
            val.fill_(-1)
            flow.fill_(-1)
            cutw.fill_(-1)
            torch.cuda.synchronize()
            rc = fn(g.n, csr.m, row.data_ptr(), head.data_ptr(), cap.data_ptr(), rev.data_ptr(), g.s, g.t,
                    val.data_ptr(), flow.data_ptr(), cutw.data_ptr(), ctypes.c_void_p(stream.cuda_stream))
            assert rc == 0, mf.lib().mf_last_error()
            torch.cuda.synchronize()
            assert int(val.item()) == ref.value
            cut = mf.cut_bits_to_bool(cutw.cpu().numpy().view(np.uint32), g.n)
            assert np.array_equal(cut, ref_cut)
            f_in = np.where(csr.arc_slot >= 0, flow.cpu().numpy()[np.maximum(csr.arc_slot, 0)], 0).astype(np.int64)
            assert not oracle.check_flow(g.n, g.s, g.t, g.tail, g.head, g.cap, f_in, ref.value, cut)


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
