"""State exchange through the C ABI with every kind of caller buffer: device
memory, pinned host memory (uploaded by DMA through device staging, or read
and written in place by a kernel) and
pageable host memory (2-D copies), including buffers that are not 16-byte
aligned."""
import numpy as np
import pytest

from paper_1308_3290_gb300 import inputs, qg
from tests.gpu_util import require_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_state_round_trip_all_buffer_kinds(dtype):
    torch = require_gpu()
    nx, ny = 64, 128
    td = torch.float32 if dtype == "f32" else torch.float64
    w = inputs.perturbation(nx, ny, seed=21)
    b = qg.Basin(nx, ny, Re=200.0, Ro=0.0016, levels=1, dt=1e-4, dtype=dtype)
    ref = torch.as_tensor(w, dtype=td)
    kinds = {
        "device": lambda: ref.to("cuda").contiguous(),
        "pinned": lambda: ref.clone().pin_memory(),
        "pageable": lambda: ref.clone(),
    }
    for name, make in kinds.items():
        src = make()
        qg.qg_set_state(b.h, src, 0)
        for out_kind in ("device", "pinned", "pageable"):
            if out_kind == "device":
                out = torch.empty_like(ref, device="cuda")
            elif out_kind == "pinned":
                out = torch.empty_like(ref).pin_memory()
            else:
                out = torch.empty_like(ref)
            qg.qg_get_state(b.h, out, 0)
            b.synchronize()
            assert torch.equal(out.cpu(), ref), (name, out_kind)
    # a pinned buffer whose start is not 16-byte aligned (scalar path)
    big = torch.empty(ref.numel() + 1, dtype=td).pin_memory()
    view = big[1:].view(ref.shape)
    view.copy_(ref)
    qg.qg_set_state(b.h, view, 0)
    out = torch.empty(ref.numel() + 1, dtype=td).pin_memory()
    outv = out[1:].view(ref.shape)
    qg.qg_get_state(b.h, outv, 0)
    b.synchronize()
    assert torch.equal(outv, ref)
    b.close()


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_get_state_async_into_pinned_buffers(dtype):
    """qg_get_state_async into page-locked buffers (aligned and not): the
    buffer holds the state after qg_synchronize; other buffers take the
    ordinary path."""
    torch = require_gpu()
    nx, ny = 64, 128
    td = torch.float32 if dtype == "f32" else torch.float64
    ref = torch.as_tensor(inputs.perturbation(nx, ny, seed=22), dtype=td)
    b = qg.Basin(nx, ny, Re=200.0, Ro=0.0016, levels=1, dt=1e-4, dtype=dtype)
    b.set_state(ref.to("cuda"))
    for out in (torch.empty_like(ref).pin_memory(),
                torch.empty(ref.numel() + 1, dtype=td).pin_memory()[1:].view(ref.shape),
                torch.empty_like(ref, device="cuda"), torch.empty_like(ref)):
        qg.qg_get_state_async(b.h, out, 0)
        b.synchronize()
        assert torch.equal(out.cpu(), ref)
    b.close()


def test_pipelined_host_exchange_matches_the_synchronous_path():
    """A different host input every step (uploaded by DMA through the two
    staging buffers while the step before computes), one step, and the
    result downloaded asynchronously into a page-locked buffer of its own:
    after one qg_synchronize every result equals, bitwise, the synchronous
    exchange through device buffers."""
    torch = require_gpu()
    nx, ny, K = 128, 256, 9
    ins = [torch.as_tensor(inputs.perturbation(nx, ny, seed=50 + k) * 30.0,
                           dtype=torch.float32).pin_memory() for k in range(K)]
    outs = [torch.empty_like(ins[0]).pin_memory() for _ in range(K)]
    b = qg.Basin(nx, ny, Re=200.0, Ro=0.0016, levels=2, dt=2e-5, dtype="f32")
    for k in range(K):
        qg.qg_set_state(b.h, ins[k], 0)
        qg.qg_step(b.h, 1)
        qg.qg_get_state_async(b.h, outs[k], 0)
    b.synchronize()
    for k in range(K):
        b.set_state(ins[k].to("cuda"))
        b.step(1)
        want = b.state().cpu()
        assert torch.equal(outs[k], want), k
    b.close()
