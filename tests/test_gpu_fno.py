"""The surrogate's GPU kernels (scw_surrogate_*) against the FP64 oracle (oracle/fno.py).

FP32 mode runs every step in FP32 on SIMT cores: loss, every gradient group and
the inferred field must match the oracle to rel-L2 <= 1e-5. BF16 mode keeps
activations and weights in BF16 and runs the DFT contractions on tcgen05:
rel-L2 <= 2e-2 per gradient group and per field. Shapes span several GEMM tiles
with ragged tails (B C = 96 and 160 rows, 4-sample weight-gradient groups with
missing samples) and the full surrogate size (64^2 grid, 16^2 modes, 4 layers).
"""
import numpy as np
import pytest

import workloads as wl
from helpers import fno_init_groups, rel_l2
from oracle import fno

pytestmark = pytest.mark.gpu

SMALL = fno.FnoShape(width=32, grid=16, modes=4, layers=3, slices=2, in_grid=8)
FULL = fno.FnoShape(width=32, grid=64, modes=16, layers=4, slices=8, in_grid=32)
TOL = {"fp32": 1e-5, "bf16": 2e-2}


def _case(sh, B, seed):
    flat = wl.random_flat(seed, fno_init_groups(sh)).astype(np.float32)
    n = wl.phantom_batch(1000 + seed, B, nx=sh.in_grid, ny=sh.in_grid, nz=sh.slices,
                         semi_axes=(1.0, sh.in_grid / 4)).astype(np.complex64)
    rng = np.random.default_rng(seed + 99)
    E = (rng.standard_normal((B, 3, sh.grid, sh.grid)) + 1j * rng.standard_normal((B, 3, sh.grid, sh.grid)))
    return flat, n, E.astype(np.complex64)


def _surrogate(sh, B, precision):
    import paper_2404_07293_gb300 as scw
    return scw.Surrogate(grid=sh.grid, modes=sh.modes, layers=sh.layers, slices=sh.slices, in_grid=sh.in_grid,
                         batch_max=B, precision=precision)


def _groups(sh):
    off = 0
    for name, s, cplx in fno.param_layout(sh):
        size = int(np.prod(s)) * (2 if cplx else 1)
        yield name, off, size
        off += size


def _compare_grads(got, ref, sh, tol):
    worst = {}
    for name, off, size in _groups(sh):
        a, b = got[off:off + size], ref[off:off + size]
        worst[name] = float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))
    print("grad rel-L2 per group", worst)
    bad = {k: v for k, v in worst.items() if v > tol}
    assert not bad, bad


@pytest.mark.parametrize("precision,B", [("fp32", 3), ("fp32", 5), ("bf16", 3), ("bf16", 5)])
def test_loss_and_gradients_match_oracle(precision, B, cuda_device):
    import torch
    sh = SMALL
    flat, n, E = _case(sh, B, seed=B)
    s = _surrogate(sh, B, precision)
    s.set_params(flat)
    nd = torch.from_numpy(n).to(cuda_device)
    Ed = torch.from_numpy(E).to(cuda_device)
    loss = s.forward_backward(nd, Ed)
    g = s.grads().astype(np.float64)
    L, Lf, Lh, gref = fno.loss_and_grads(flat.astype(np.float64), n.astype(np.complex128),
                                          fno.channels_from_field(E.astype(np.complex128)), sh)
    print(precision, "loss", loss, "oracle", (L, Lf, Lh))
    tol = TOL[precision]
    assert abs(loss[1] - Lf) <= tol * abs(Lf) and abs(loss[2] - Lh) <= tol * max(abs(Lh), 1.0)
    _compare_grads(g, gref, sh, tol)
    s.close()


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_inference_matches_oracle(precision, cuda_device):
    import torch
    sh, B = SMALL, 5
    flat, n, _ = _case(sh, B, seed=11)
    s = _surrogate(sh, B, precision)
    s.set_params(flat)
    field, est, flag = s.infer(torch.from_numpy(n).to(cuda_device), threshold=0.5)
    torch.cuda.synchronize()
    Fref, href, _ = fno.forward(flat.astype(np.float64), n.astype(np.complex128), sh)
    ref = fno.field_from_channels(Fref)
    got = field.cpu().numpy()
    for b in range(B):
        err = max(rel_l2(got[b], ref[b]))
        assert err <= TOL[precision], (b, err)
    h = np.log(est.cpu().numpy().astype(np.float64))
    assert np.abs(h - href).max() <= (1e-4 if precision == "fp32" else 5e-2)
    assert np.array_equal(flag.cpu().numpy().astype(bool), np.exp(h) > 0.5)
    s.close()


def test_full_size_bf16_against_oracle(cuda_device):
    """64^2 grid, 16^2 modes, 4 layers, 8 slices of 32^2; 6 samples (two 4-sample
    weight-gradient groups, the second ragged)."""
    import torch
    sh, B = FULL, 6
    flat, n, E = _case(sh, B, seed=21)
    s = _surrogate(sh, B, "bf16")
    s.set_params(flat)
    nd, Ed = torch.from_numpy(n).to(cuda_device), torch.from_numpy(E).to(cuda_device)
    field, _, _ = s.infer(nd)
    torch.cuda.synchronize()
    Fref, _, _ = fno.forward(flat.astype(np.float64), n.astype(np.complex128), sh)
    ref = fno.field_from_channels(Fref)
    got = field.cpu().numpy()
    errs = [max(rel_l2(got[b], ref[b])) for b in range(B)]
    print("full-size field rel-L2", errs)
    assert max(errs) <= TOL["bf16"]
    s.forward_backward(nd, Ed)
    g = s.grads().astype(np.float64)
    _, _, _, gref = fno.loss_and_grads(flat.astype(np.float64), n.astype(np.complex128),
                                       fno.channels_from_field(E.astype(np.complex128)), sh)
    _compare_grads(g, gref, sh, TOL["bf16"])
    s.close()


def test_train_step_is_one_adam_step(cuda_device):
    import torch
    sh, B = SMALL, 4
    flat, n, E = _case(sh, B, seed=31)
    s = _surrogate(sh, B, "fp32")
    s.set_params(flat)
    nd, Ed = torch.from_numpy(n).to(cuda_device), torch.from_numpy(E).to(cuda_device)
    s.train_step(nd, Ed, lr=1e-3)
    got = s.params().astype(np.float64)
    g = s.grads().astype(np.float64)
    ref, _, _ = fno.adam_step(flat.astype(np.float64), g, np.zeros_like(g), np.zeros_like(g), 1, 1e-3)
    assert np.abs(got - ref).max() <= 1e-6
    s.close()


def test_training_reduces_loss_on_a_teacher_network(cuda_device):
    """A student (BF16 kernels, Adam) fits the field of a random teacher network
    of the same architecture: the loss falls well below its start."""
    import torch
    sh, B = fno.FnoShape(width=32, grid=32, modes=8, layers=2, slices=4, in_grid=16), 16
    teacher = wl.random_flat(7, fno_init_groups(sh))
    n_all = wl.phantom_batch(500, 64, nx=sh.in_grid, ny=sh.in_grid, nz=sh.slices, semi_axes=(1.0, 4.0))
    F, _, _ = fno.forward(teacher, n_all, sh)
    T_all = fno.field_from_channels(F).astype(np.complex64)
    s = _surrogate(sh, B, "bf16")
    s.set_params(wl.random_flat(8, fno_init_groups(sh)).astype(np.float32))
    nd = torch.from_numpy(n_all.astype(np.complex64)).to(cuda_device)
    Td = torch.from_numpy(T_all).to(cuda_device)
    losses = []
    for step in range(300):
        i = (step * B) % 64
        losses.append(s.train_step(nd[i:i + B].contiguous(), Td[i:i + B].contiguous(), lr=2e-3)[1])
    print("field loss start", losses[:3], "end", losses[-3:])
    assert np.mean(losses[-10:]) < 0.2 * np.mean(losses[:3])
    s.close()


def test_calibration_matches_conformal_rule(cuda_device):
    import paper_2404_07293_gb300 as scw  # noqa: F401
    sh = SMALL
    s = _surrogate(sh, 2, "fp32")
    rng = np.random.default_rng(3)
    est = np.exp(rng.normal(-3, 1, 200)).astype(np.float32)
    true = (est * np.exp(rng.normal(0, 0.5, 200))).astype(np.float32)
    q = s.calibrate(est, true, miss=0.05)
    ref = fno.conformal_offset(np.log(est.astype(np.float64)), true.astype(np.float64), 0.05)
    assert q == pytest.approx(ref, abs=1e-5)
    s.close()


def test_backward_with_several_tiles_per_cta_matches_half_batches(cuda_device):
    """Full size at 320 samples: the backward DFT + weight-gradient kernel then has 160 tiles for at
    most 152 CTAs, so some CTAs run two tiles through their single accumulator pair. The loss is a
    mean over samples, so the gradient of the 320-sample batch is the mean of the gradients of its
    two 160-sample halves (80 tiles: one per CTA). Per-sample arithmetic is the same in both, only
    the sums over samples are grouped differently."""
    import torch
    sh, B = FULL, 320
    flat, n, E = _case(sh, B, seed=33)
    grads = []
    for lo, hi in ((0, B), (0, B // 2), (B // 2, B)):
        s = _surrogate(sh, hi - lo, "bf16")
        s.set_params(flat)
        nd = torch.from_numpy(np.ascontiguousarray(n[lo:hi])).to(cuda_device)
        Ed = torch.from_numpy(np.ascontiguousarray(E[lo:hi])).to(cuda_device)
        s.forward_backward(nd, Ed)
        torch.cuda.synchronize()
        grads.append(s.grads().astype(np.float64))
        s.close()
    whole, half = grads[0], 0.5 * (grads[1] + grads[2])
    _compare_grads(whole, half, sh, 1e-4)
