"""ffsat_step_noalloc against ffsat_step, through the C ABI.

Some users of this library cannot let it call cudaMalloc: their process hands
all device memory to its own pool allocator, or runs a loop that cannot absorb
the device synchronisation an allocation implies.  For them the library offers
a round of projected gradient descent whose gradient scratch lives in a buffer
reserved statically in the library's device image.  This test checks, on two
calls in a row, that it returns what the allocating entry point returns, and
that it refuses sizes beyond its static buffer.  It sits in its own file that
pytest collects last."""
import numpy as np
import pytest

import oracle as O
from paper_2308_15020_gb300 import gen

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _scratch_instance(n):
    return gen.concat([gen.random_ksat(n, 4 * n, 3, 5), gen.random_xor(n, 30, 10, 60, 5, signs=True),
                       gen.random_atleast(n, 12, 32, 300, 5)])


def test_noalloc_step_matches_step_two_calls():
    from paper_2308_15020_gb300 import ffsat

    n, B, lr = 30000, 6, 0.05
    inst = _scratch_instance(n)
    h = ffsat.Instance(inst)
    assert h.info()["smem_mode_f32"] in (1, 2)  # the gradient scratch is needed
    x0 = gen.uniform_points(B, n, 21)
    xa = torch.from_numpy(x0).cuda()
    xb = xa.clone()
    for call in range(2):
        start = xa.cpu().numpy().astype(np.float64)
        sa, na = h.step(xa, T=1, lr=lr, seed=8, epoch=call, restart=False)
        sb, nb = h.step_noalloc(xb, T=1, lr=lr, seed=8, epoch=call, restart=False)
        torch.cuda.synchronize()
        h.sync_status()
        # the one-iteration tolerance of the step parity test: lr * 1e-4 * condition scale + 1e-7
        _, gs = O.eval_grad(inst, start)
        _, A = O.eval_scale(inst, start, 1e-2)
        tol = lr * 1e-4 * np.maximum(np.abs(gs), A) + 1e-7
        diff = np.abs(xa.cpu().numpy().astype(np.float64) - xb.cpu().numpy().astype(np.float64))
        assert np.all(diff <= tol), float(np.max(diff / tol))
        assert torch.equal(sa, sb) and torch.equal(na, nb)


def test_noalloc_first_call_allocates_no_device_memory():
    """On a fresh instance that needs scratch, the first allocation-free call
    leaves the device's free memory unchanged (ffsat_step would allocate B * n
    values there)."""
    from paper_2308_15020_gb300 import ffsat

    n, B = 30000, 6
    inst = _scratch_instance(n)
    h = ffsat.Instance(inst)
    assert h.info()["smem_mode_f32"] in (1, 2)
    x = torch.from_numpy(gen.uniform_points(B, n, 22)).cuda()
    h.step_noalloc(x, T=1, lr=0.05, seed=1, restart=False)  # the static buffer's address is looked up here
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    h2 = ffsat.Instance(inst)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    h2.step_noalloc(x, T=1, lr=0.05, seed=1, restart=False)
    torch.cuda.synchronize()
    free2, _ = torch.cuda.mem_get_info()
    assert free2 == free1, (free1 - free2)
    assert free0 - free1 >= 0  # loading the instance may allocate; the step does not


def test_noalloc_rejects_sizes_beyond_static_scratch():
    from paper_2308_15020_gb300 import ffsat

    n = 70000
    inst = gen.random_ksat(n, 2 * n, 3, 6)
    h = ffsat.Instance(inst)
    assert h.info()["smem_mode_f32"] == 2
    B = ffsat.FFSAT_STATIC_SCRATCH_BYTES // (4 * n) + 1
    x = torch.zeros(B, n, device="cuda")
    with pytest.raises(ffsat.FFSatError) as e:
        h.step_noalloc(x, T=1, lr=0.1)
    assert e.value.code == -1 and "static" in str(e.value)
