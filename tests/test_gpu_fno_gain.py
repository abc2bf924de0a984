"""What the trained surrogate gains over the plain method without it.

Targets are exit-plane fields of seeded ellipsoid phantoms (32x32x8 voxels of
0.25 um, lambda = 1 um, normally incident x-polarised plane wave) computed by
the FP64 coupled-wave oracle at 7x7 orders, so that the whole test, data
included, runs in about a minute. The surrogate (4 Fourier layers, width 32,
16x16 modes, 64x64 output) trains on the GPU with its own BF16 kernels.
Periodic lateral shifts of a sample shift its exit field (normal incidence on a
periodic sample), so each batch is shifted by a random whole number of voxels.

Without the learned part, every field needs a solve; the best field-free guess
(the mean training field) is what the method offers without solving. The test
checks that the trained network
  - predicts held-out fields far better than that guess,
  - is orders of magnitude faster than the plain method on the GPU at the same
    orders (scw_solve + recomposition of the exit field, timed here on the
    held-out seeds, whose fields also agree with the oracle's),
  - has an error head whose estimates track the true error, and
  - after split-conformal calibration, accepts samples whose true error is
    mostly below the threshold (the rest fall back to the plain method).
"""
import numpy as np
import pytest

import fno_data

pytestmark = pytest.mark.gpu

N_TRAIN, N_CAL, N_TEST = 640, 64, 64
THRESHOLD = 0.2


def _rel(a, b):
    return np.sqrt((np.abs(a - b) ** 2).sum(axis=(1, 2, 3)) / (np.abs(b) ** 2).sum(axis=(1, 2, 3)))


def test_surrogate_gain_over_plain_method(cuda_device):
    import time

    import torch
    import paper_2404_07293_gb300 as scw

    seeds = list(range(N_TRAIN + N_CAL)) + list(range(500_000, 500_000 + N_TEST))
    n, E, solve_s = fno_data.exit_fields(seeds, U=7)
    ntr, Etr = n[:N_TRAIN], E[:N_TRAIN]
    ncal, Ecal = n[N_TRAIN:N_TRAIN + N_CAL], E[N_TRAIN:N_TRAIN + N_CAL]
    nte, Ete = n[N_TRAIN + N_CAL:], E[N_TRAIN + N_CAL:]

    dev = cuda_device
    s = scw.Surrogate(grid=64, modes=16, layers=4, slices=8, in_grid=32, batch_max=64, precision="bf16", seed=3)
    nd, Ed = torch.from_numpy(ntr).to(dev), torch.from_numpy(Etr).to(dev)
    g = torch.Generator(device="cpu").manual_seed(0)
    steps, B = 2000, 32
    first = last = None
    for st in range(steps):
        idx = torch.randint(0, N_TRAIN, (B,), generator=g).to(dev)
        dy, dx = (int(v) for v in torch.randint(0, 32, (2,), generator=g))
        nb = torch.roll(nd[idx], shifts=(dy, dx), dims=(2, 3)).contiguous()
        Eb = torch.roll(Ed[idx], shifts=(2 * dy, 2 * dx), dims=(2, 3)).contiguous()
        lr = 1e-3 if st < 0.8 * steps else 1e-4
        read = st == 0 or st >= steps - 20
        loss = s.train_step(nb, Eb, lr=lr, read_loss=read)
        if st == 0:
            first = loss[1]
        elif read:
            last = loss[1] if last is None else min(last, loss[1])

    field, _, _ = s.infer(torch.from_numpy(nte).to(dev))
    err = _rel(field.cpu().numpy(), Ete)
    guess = _rel(np.broadcast_to(Etr.mean(0, keepdims=True), Ete.shape), Ete)

    # calibrate the error head on the calibration split, then gate the held-out split
    fc, est_cal, _ = s.infer(torch.from_numpy(ncal).to(dev))
    err_cal = _rel(fc.cpu().numpy(), Ecal)
    q = s.calibrate(est_cal.cpu().numpy(), err_cal, miss=0.1)
    s.set_offset(q)
    nte_d = torch.from_numpy(nte).to(dev)
    _, est, flag = s.infer(nte_d, threshold=THRESHOLD)
    est, flag = est.cpu().numpy(), flag.cpu().numpy().astype(bool)
    corr = np.corrcoef(np.log(est), np.log(err))[0, 1]
    accepted = ~flag
    violations = float(np.mean(err[accepted] > THRESHOLD)) if accepted.any() else 0.0

    # the plain method on the GPU at the same orders, on the held-out seeds (two solves in flight,
    # after a warm-up that creates the solvers' library handles)
    fno_data.exit_fields_gpu(seeds[-2:], U=7, workers=2)
    t0 = time.perf_counter()
    _, E_gpu, _ = fno_data.exit_fields_gpu(seeds[-N_TEST:], U=7, workers=2)
    plain_per_sample = (time.perf_counter() - t0) / N_TEST
    assert _rel(E_gpu, Ete).max() <= 1e-5

    # speed: one batched inference against the plain method per sample
    for _ in range(3):
        s.infer(nte_d)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(20):
        s.infer(nte_d)
    torch.cuda.synchronize()
    per_sample = (time.perf_counter() - t0) / 20 / N_TEST
    speedup = plain_per_sample / per_sample
    s.close()

    print(f"train field loss {first:.3f} -> {last:.2e}; held-out rel-L2 median {np.median(err):.3f} "
          f"(max {err.max():.3f}) vs mean-field guess {np.median(guess):.3f}; head log-corr {corr:.2f}; "
          f"q {q:.2f}; accepted {accepted.mean():.2f} at threshold {THRESHOLD} with {violations:.2f} above it; "
          f"inference {per_sample * 1e6:.1f} us/sample vs the GPU plain method {plain_per_sample * 1e3:.2f} ms/sample "
          f"({speedup:.2e}x; the FP64 oracle solve takes {np.mean(solve_s):.3f} s)")
    assert last < 0.05 * first
    assert np.median(err) < 0.35 * np.median(guess)
    assert speedup > 1e3
    assert corr > 0.3
    assert violations <= 0.25
