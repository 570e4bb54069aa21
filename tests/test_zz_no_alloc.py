"""The allocation-free RMSE entry point (std_rmse_static).

It serves callers that cannot let the library allocate device memory (a
process whose device memory is held by its own pool, or a loop that cannot
afford cudaMalloc/cudaFree, which synchronises the device).  Its scratch is a
fixed array inside the library shared by every call, so this test calls it
twice in a row, with different sizes, and checks each result against the
context's std_rmse within the tolerance of the RMSE parity tests (1e-5
relative).  This file is collected last on purpose.
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
    cases = [(tc.shape[0], dc, dv, want_full), (sub, dc[:sub], dv[:sub], want_sub),
             (tc.shape[0], dc, dv, want_full)]
    for k, cc, vv, want in cases:
        out.fill_(-1.0)
        B.std_rmse_static(3, shape, ranks, R, dA, dB, k, cc, vv, out, stream.cuda_stream)
        stream.synchronize()
        got = out.cpu().numpy()
        assert abs(got[0] - want[0]) <= 1e-5 * want[0], (got, want)
        assert abs(got[1] - want[1]) <= 1e-5 * want[1], (got, want)

    # k = 0 writes {0, 0}; a size beyond the limits is refused
    out.fill_(-1.0)
    B.std_rmse_static(3, shape, ranks, R, dA, dB, 0, dc, dv, out, stream.cuda_stream)
    stream.synchronize()
    assert out.cpu().tolist() == [0.0, 0.0]
    with pytest.raises(B.StdError) as ei:
        B.std_rmse_static(3, shape, ranks, 64, dA, dB, 10, dc, dv, out, stream.cuda_stream)
    assert ei.value.code == B.STD_EUNSUPPORTED
