"""The allocation-free RMSE entry point (std_rmse_static).

It serves callers that cannot let the library allocate device memory (a
process whose device memory is held by its own pool, or a loop that cannot
afford cudaMalloc/cudaFree, which synchronises the device).  Its scratch is a
fixed array inside the library shared by every call, so this test calls it
twice in a row, with different sizes, and checks each result against the
context's std_rmse within the tolerance of the RMSE parity tests (1e-5
relative) and against the FP64 oracle's RMSE/MAE of the same FP32 model; it
also checks that a call after the first allocates no device memory, and that
an out-of-range coordinate gives NaN without being read through.  This file
is collected last on purpose.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_rmse_static_matches_std_rmse_on_consecutive_calls():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import __graft_entry__ as ge
    ge.build()
    from paper_2012_03550_gb300 import binding as B
    from paper_2012_03550_gb300 import synth

    w = synth.config1()
    c, v = w.tensor.split("train")
    tc, tv = w.tensor.split("test")
    shape, ranks, R = w.tensor.shape, w.ranks, w.r_core
    A0, B0 = synth.init_params(shape, ranks, R, mode="normal", seed=1)
    sub = 1234
    with B.Tucker(shape, ranks, c, v, r_core=R) as g:
        g.set_params(A0, B0, epoch=0)
        g.epoch(0.5, 0.5, w.lam, w.lam, w.minibatch)
        want_full = g.rmse(tc, tv)
        want_sub = g.rmse(tc[:sub], tv[:sub])
        A1, B1, _, _ = g.get_params()

    dev = torch.device("cuda", torch.cuda.current_device())
    dA = [torch.from_numpy(a).to(dev) for a in A1]
    dB = [torch.from_numpy(b).to(dev) for b in B1]
    dc = torch.from_numpy(tc).to(dev)
    dv = torch.from_numpy(tv).to(dev)
    out = torch.empty(2, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    from oracle import oracle as O
    ref = O.Model(shape, ranks, R, A1, B1)
    ref.build_core()
    orc_full = ref.rmse_mae(tc, tv)
    orc_sub = ref.rmse_mae(tc[:sub], tv[:sub])
    cases = [(tc.shape[0], dc, dv, want_full, orc_full), (sub, dc[:sub], dv[:sub], want_sub, orc_sub),
             (tc.shape[0], dc, dv, want_full, orc_full)]
    for i, (k, cc, vv, want, orc) in enumerate(cases):
        out.fill_(-1.0)
        if i == 1:
            torch.cuda.synchronize()
            alloc0 = torch.cuda.memory_allocated(dev)
            free0 = torch.cuda.mem_get_info(dev)[0]
        B.std_rmse_static(3, shape, ranks, R, dA, dB, k, cc, vv, out, stream.cuda_stream)
        stream.synchronize()
        if i == 1:
            # after the first call (which may load the module and look up the
            # scratch address) a call takes no device memory at all
            assert torch.cuda.memory_allocated(dev) == alloc0
            assert torch.cuda.mem_get_info(dev)[0] == free0
        got = out.cpu().numpy()
        assert abs(got[0] - want[0]) <= 1e-5 * want[0], (got, want)
        assert abs(got[1] - want[1]) <= 1e-5 * want[1], (got, want)
        # the FP32 model's RMSE/MAE in FP64 (Eq. 19): FP32 predictions differ
        # from the oracle's FP64 ones by a few ulps of x-hat
        assert abs(got[0] - orc[0]) <= 1e-5 * orc[0], (got, orc)
        assert abs(got[1] - orc[1]) <= 1e-5 * orc[1], (got, orc)

    # a coordinate equal to I_n is checked before any read: both results NaN
    bad = dc[:16].clone()
    bad[5, 1] = shape[1]
    out.fill_(-1.0)
    B.std_rmse_static(3, shape, ranks, R, dA, dB, 16, bad, dv[:16], out, stream.cuda_stream)
    stream.synchronize()
    assert np.isnan(out.cpu().numpy()).all()

    # k = 0 writes {0, 0}; a size beyond the limits is refused
    out.fill_(-1.0)
    B.std_rmse_static(3, shape, ranks, R, dA, dB, 0, dc, dv, out, stream.cuda_stream)
    stream.synchronize()
    assert out.cpu().tolist() == [0.0, 0.0]
    # the library's own limit check (the binding's shape checks would stop
    # this call first, so the library is called directly)
    import ctypes
    ms = np.ascontiguousarray(shape, dtype=np.int64)
    rk = np.ascontiguousarray(ranks, dtype=np.int32)
    rc = B.lib().std_rmse_static(3, ms.ctypes.data, rk.ctypes.data, 64, B._ptr_array(dA), B._ptr_array(dB), 10,
                                 dc.data_ptr(), dv.data_ptr(), out.data_ptr(), ctypes.c_void_p(stream.cuda_stream))
    assert rc == B.STD_EUNSUPPORTED
    with pytest.raises(ValueError):
        B.std_rmse_static(3, shape, ranks, 64, dA, dB, 10, dc, dv, out, stream.cuda_stream)
