"""jko_step_noalloc: the step for callers that cannot allocate device memory.

Such callers (code inside a framework that owns all device memory through its
own pool, where a cudaMalloc escapes the pool and a cudaFree synchronises the
device; services that forbid allocation after start-up) get a step whose
working buffers live in one fixed device array inside the library.  This
checks it through the C ABI against jko_step on the same inputs, on two calls
in a row with different energies (a stale scratch would show in the second).
The file is collected last on purpose."""
import numpy as np
import pytest

from paper_1502_06216_gb300 import inputs
from tests.gpu_util import need_gpu, rel_l1

pytestmark = pytest.mark.gpu


def test_noalloc_matches_jko_step_on_two_calls():
    torch = need_gpu()
    from paper_1502_06216_gb300 import jko
    cases = [
        inputs.config_problem(1, n=96, ny=80, tol=1e-6, max_iter=300),   # porous + obstacles
        inputs.config_problem(0, n=64, tol=1e-6),                         # crowd motion
    ]
    for pb in cases:
        h = jko.create_from_problem(pb, precision=jko.Precision.FP32)
        q = torch.tensor(pb.q0, dtype=torch.float32, device="cuda")
        ref, info_ref = jko.jko_step(h, q)
        out = torch.full_like(q, -1.0)
        status, info = jko.jko_step_noalloc(pb, q, out)
        torch.cuda.synchronize()
        err = rel_l1(out.double().cpu().numpy(), ref.double().cpu().numpy())
        print(pb.name, "noalloc vs jko_step rel L1:", err, "iters", info["iters"], info_ref["iters"])
        assert status == jko.Status(info_ref["status"])
        assert err <= 1e-5
        assert info["iters"] == info_ref["iters"]
        jko.jko_destroy(h)


def test_noalloc_rejects_grids_beyond_its_scratch():
    torch = need_gpu()
    from paper_1502_06216_gb300 import jko
    pb = inputs.config_problem(0, n=257)
    q = torch.tensor(pb.q0, dtype=torch.float32, device="cuda")
    out = torch.full_like(q, -1.0)
    with pytest.raises(jko.JKOError) as e:
        jko.jko_step_noalloc(pb, q, out)
    assert e.value.status == jko.Status.UNSUPPORTED
    assert torch.all(out == -1.0)
