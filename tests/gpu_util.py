"""Helpers of the GPU tests: device buffers from torch, oracle comparisons."""
import numpy as np


def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU test needs CUDA"
    return torch


def rrsvd_device(B, plan, theta, chain0=0, want_uv=True):
    """Runs rrsvd_execute on device buffers; returns numpy results.  theta is
    a host array, or a contiguous complex128 tensor already on the device."""
    torch = torch_cuda()
    batch, m, n = theta.shape
    k, l = B.rrsvd_plan_dims(plan)
    dev = torch.device("cuda:0")
    if isinstance(theta, torch.Tensor):
        assert theta.is_cuda and theta.is_contiguous() and theta.dtype == torch.complex128
        th = theta
    else:
        th = torch.from_numpy(np.ascontiguousarray(theta)).to(dev)
    sg = torch.zeros((batch, k), dtype=torch.float64, device=dev)
    U = torch.zeros((batch, m, k), dtype=torch.complex128, device=dev) if want_uv else None
    Vh = torch.zeros((batch, k, n), dtype=torch.complex128, device=dev) if want_uv else None
    w = torch.zeros(batch, dtype=torch.float64, device=dev)
    rk = torch.zeros(batch, dtype=torch.int32, device=dev)
    wsb = B.rrsvd_workspace_size(plan)
    ws = torch.empty(wsb + 256, dtype=torch.uint8, device=dev)
    base = ws.data_ptr()
    base = (base + 255) // 256 * 256
    st = torch.cuda.current_stream().cuda_stream
    B.rrsvd_execute(plan, th.data_ptr(), chain0, sg.data_ptr(), U.data_ptr() if want_uv else 0,
                    Vh.data_ptr() if want_uv else 0, w.data_ptr(), rk.data_ptr(), base, wsb, st)
    torch.cuda.synchronize()
    out = {"sigma": sg.cpu().numpy(), "w": w.cpu().numpy(), "rank": rk.cpu().numpy(), "k": k, "l": l}
    if want_uv:
        out["U"] = U.cpu().numpy()
        out["Vh"] = Vh.cpu().numpy()
    return out


def truncated(U, s, Vh):
    return (U * s[None, :]) @ Vh


def repeat_on_device(base, batch):
    """A batch of `batch` matrices on the device, instance t = base[t % len(base)]
    (full-size batches without holding every copy in host memory)."""
    torch = torch_cuda()
    b = torch.from_numpy(np.ascontiguousarray(np.stack(base))).to("cuda:0")
    idx = torch.arange(batch, device=b.device) % len(base)
    return b[idx].contiguous()
