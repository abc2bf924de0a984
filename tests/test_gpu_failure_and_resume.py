"""Failure detection and checkpoint/resume on the GPU, without faulting it.

- Every spin-wait of the tensor-core contraction is bounded by a %globaltimer
  deadline. With stall injection on, one CTA waits on a stage that nothing
  fills (its producer skips it); after the plan's 5 ms timeout the kernel
  records the failure in the plan's device error word, lets its issued copies
  and MMAs land, frees its tensor memory and returns. scw_plan_check then
  reports SCW_ERR_TIMEOUT; the same plan without injection synthesises the
  exact field again.
- The surrogate's training state saved after some steps, loaded into a fresh
  handle, gives a next Adam step bit-identical to the original handle's.
"""
import numpy as np
import pytest

import workloads as wl
from helpers import fno_init_groups
from oracle import fno

pytestmark = pytest.mark.gpu


def test_contraction_timeout_is_reported_and_plan_recovers(cuda_device):
    import torch
    import paper_2404_07293_gb300 as scw
    U, L = 15, 8
    W, g, a, *_ = wl.random_layer_set(3, U, U, L)
    zb = np.linspace(0.0, 2.0, L + 1)
    zp = wl.cell_centred_planes(0.0, 2.0, 32 * L)
    plan = scw.Plan(U, U, L, 1.0, 4.0, 4.0, zb, 64, 64, zp, precision="split_bf16")
    plan.set_layers(torch.from_numpy(W).to(cuda_device), torch.from_numpy(g).to(cuda_device),
                    torch.from_numpy(a).to(cuda_device))
    ref = plan.synthesize().clone()
    plan.check()

    plan.set_timeout_ns(5_000_000)
    plan.inject_stall(True)
    plan.synthesize()
    with pytest.raises(scw.ScwError) as err:
        plan.check()
    assert err.value.status == 5  # SCW_ERR_TIMEOUT

    plan.inject_stall(False)
    plan.set_timeout_ns(2_000_000_000)
    again = plan.synthesize()
    plan.check()
    assert torch.equal(again, ref)
    plan.close()


@pytest.mark.parametrize("precision", ["bf16", "fp32"])
def test_surrogate_resume_is_bit_identical(precision, tmp_path, cuda_device):
    import torch
    import paper_2404_07293_gb300 as scw
    sh = fno.FnoShape(width=32, grid=16, modes=4, layers=2, slices=2, in_grid=8)
    B = 4
    n = torch.from_numpy(wl.phantom_batch(9, B, nx=8, ny=8, nz=2, semi_axes=(1.0, 2.0)).astype(np.complex64))
    rng = np.random.default_rng(4)
    T = torch.from_numpy((rng.standard_normal((B, 3, 16, 16)) + 1j * rng.standard_normal((B, 3, 16, 16)))
                         .astype(np.complex64))
    n, T = n.to(cuda_device), T.to(cuda_device)
    kw = dict(grid=16, modes=4, layers=2, slices=2, in_grid=8, batch_max=B, precision=precision)
    a = scw.Surrogate(**kw)
    a.set_params(wl.random_flat(1, fno_init_groups(sh)).astype(np.float32))
    for _ in range(5):
        a.train_step(n, T, lr=3e-3)
    a.set_offset(0.25)
    path = tmp_path / "state.pt"
    a.save(path)
    a.train_step(n, T, lr=3e-3)
    after_a = a.params()

    b = scw.Surrogate(**kw)
    b.load(path)
    b.train_step(n, T, lr=3e-3)
    after_b = b.params()
    assert np.array_equal(after_a, after_b)
    _, est_a, _ = a.infer(n)
    _, est_b, _ = b.infer(n)
    torch.cuda.synchronize()
    assert torch.equal(est_a, est_b)  # the calibration offset came back too

    with pytest.raises(scw.ScwError):
        b.load_state(np.zeros(16, dtype=np.uint8))
    a.close()
    b.close()
