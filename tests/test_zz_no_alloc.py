"""agp_katz_lambda_noalloc: the allocation-free lambda_1 entry point, checked through the C ABI.

It serves callers that may not allocate device memory while they run (their memory belongs to
another allocator, or cudaMalloc/cudaFree would synchronise the device under them). The test
builds a graph with the ordinary entry points (the test itself may allocate), hands the device CSR
to the no-alloc entry point twice in a row, and compares lambda_1 with agp_katz_beta's at the
tolerance the other lambda_1 test uses (relative 1e-9). The file is named to be collected last.
"""
import ctypes as C

import numpy as np
import pytest

from synth import graphs as SG

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_noalloc_lambda_matches_katz_beta_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2106_03058_gb300 as agp
    L = agp.lib()
    n = 16384
    u, v = SG.rmat_edges(n, 131072, seed=20210604)
    g = agp.build_graph(n, u, v)
    try:
        _, lam_ref = agp.katz_beta(g, 0.85, iters=5000, tol=1e-13)
        nn, nnz = C.c_int64(), C.c_int64()
        rp, ci = C.c_void_p(), C.c_void_p()
        assert L.agp_graph_info(g.handle, C.byref(nn), C.byref(nnz), C.byref(rp), C.byref(ci), None) == 0
        stream = torch.cuda.current_stream().cuda_stream
        for _ in range(2):  # the shared scratch keeps the previous call's contents
            lam = C.c_double()
            rc = L.agp_katz_lambda_noalloc(nn.value, rp.value, ci.value, 5000, 1e-13, C.byref(lam), stream)
            assert rc == 0, L.agp_last_error_detail()
            assert abs(lam.value - lam_ref) <= 1e-9 * lam_ref
        # sizes beyond the fixed scratch are refused with a message
        lam = C.c_double()
        rc = L.agp_katz_lambda_noalloc(4194305, rp.value, ci.value, 10, 1e-6, C.byref(lam), stream)
        assert rc == 1 and b"4194304" in L.agp_last_error_detail()
    finally:
        g.destroy()
