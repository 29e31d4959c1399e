"""State exchange through the C ABI with every kind of caller buffer: device
memory, pinned host memory (repacked by a kernel over the host link) and
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
