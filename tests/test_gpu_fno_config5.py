"""The learned surrogate at the orders it is specified for: 15x15.

Phantoms of 32x32x8 voxels of 0.25 um (1-8 seeded ellipsoids with semi-axes of
2-8 voxels), lambda = 1 um, a normally incident x-polarised plane wave. The
targets are exit-plane fields (64x64, just below the sample) from the plain
method on the GPU: scw_solve at 15x15 orders, then the recomposition of the
transmitted spectrum. A random subset of them is checked against the FP64
oracle's solve and direct sum. Training seeds start at 0 (the last tenth is the
calibration split of the error head), held-out seeds at 1,000,000.

The surrogate (4 Fourier layers, width 32, 16x16 modes) trains with its own
BF16 kernels; its error head is calibrated split-conformally (miss rate 5 %) and
gates the held-out samples at rel-L2 5e-2: above it a sample falls back to the
plain method. The test reports the held-out rel-L2 distribution, the acceptance
and violation rates, and the time per sample of inference against the plain
method on the same GPU.

Sizes default to a small study that finishes in a few minutes; the environment
variables SCW_C5_TRAIN (training + calibration samples), SCW_C5_TEST (held-out
samples) and SCW_C5_STEPS (Adam steps) scale it up.
"""
import json
import os
import time

import numpy as np
import pytest

import fno_data

pytestmark = pytest.mark.gpu

N_FIT = int(os.environ.get("SCW_C5_TRAIN", "160"))
N_TEST = int(os.environ.get("SCW_C5_TEST", "64"))
STEPS = int(os.environ.get("SCW_C5_STEPS", "3000"))
THRESHOLD = 5e-2
MISS = 0.05
ORACLE_CHECK = 4


def _rel(a, b):
    return np.sqrt((np.abs(a - b) ** 2).sum(axis=(1, 2, 3)) / (np.abs(b) ** 2).sum(axis=(1, 2, 3)))


def test_surrogate_at_15x15_orders_gated_at_5e_2(cuda_device):
    rng = np.random.default_rng(2024)
    n_cal = max(16, N_FIT // 10)
    n_train = N_FIT - n_cal
    fit_seeds = list(range(N_FIT))
    test_seeds = list(range(1_000_000, 1_000_000 + N_TEST))
    check_seeds = sorted(rng.choice(fit_seeds, ORACLE_CHECK // 2, replace=False).tolist() +
                         rng.choice(test_seeds, ORACLE_CHECK // 2, replace=False).tolist())
    # the oracle's spot check runs in spawned processes before any GPU work of this test
    n_o, E_o, oracle_s = fno_data.exit_fields(check_seeds, U=15, workers=ORACLE_CHECK)

    import torch
    import paper_2404_07293_gb300 as scw

    t0 = time.perf_counter()
    n_fit, E_fit, _ = fno_data.exit_fields_gpu(fit_seeds, U=15, workers=2)
    n_te, E_te, _ = fno_data.exit_fields_gpu(test_seeds, U=15, workers=2)
    gen_s = time.perf_counter() - t0
    plain_per_sample = gen_s / (N_FIT + N_TEST)  # the plain method's GPU throughput (two solves in flight)

    # targets from the GPU plain method agree with the FP64 oracle
    pos = {s: i for i, s in enumerate(fit_seeds)}
    pos_te = {s: i for i, s in enumerate(test_seeds)}
    for k, s in enumerate(check_seeds):
        E = E_fit[pos[s]] if s in pos else E_te[pos_te[s]]
        err = [float(np.linalg.norm(E[c] - E_o[k][c]) / np.linalg.norm(E_o[k][c])) for c in range(3)]
        assert max(err) <= 1e-5, (s, err)

    ntr, Etr = n_fit[:n_train], E_fit[:n_train]
    ncal, Ecal = n_fit[n_train:], E_fit[n_train:]
    dev = cuda_device
    B = 64
    s = scw.Surrogate(grid=64, modes=16, layers=4, slices=8, in_grid=32, batch_max=256, precision="bf16", seed=5)
    nd, Ed = torch.from_numpy(ntr).to(dev), torch.from_numpy(Etr).to(dev)
    g = torch.Generator(device="cpu").manual_seed(1)
    first = last = None
    t0 = time.perf_counter()
    for st in range(STEPS):
        idx = torch.randint(0, n_train, (B,), generator=g).to(dev)
        dy, dx = (int(v) for v in torch.randint(0, 32, (2,), generator=g))
        nb = torch.roll(nd[idx], shifts=(dy, dx), dims=(2, 3)).contiguous()
        Eb = torch.roll(Ed[idx], shifts=(2 * dy, 2 * dx), dims=(2, 3)).contiguous()
        lr = 1e-3 if st < 0.7 * STEPS else (3e-4 if st < 0.9 * STEPS else 1e-4)
        read = st == 0 or st >= STEPS - 20
        loss = s.train_step(nb, Eb, lr=lr, read_loss=read)
        if st == 0:
            first = loss[1]
        elif read:
            last = loss[1] if last is None else min(last, loss[1])
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0

    def infer_all(n):
        fields, ests = [], []
        for i in range(0, len(n), 256):
            f, e, _ = s.infer(torch.from_numpy(n[i:i + 256]).to(dev))
            fields.append(f.cpu().numpy())
            ests.append(e.cpu().numpy())
        return np.concatenate(fields), np.concatenate(ests)

    f_cal, est_cal = infer_all(ncal)
    err_cal = _rel(f_cal, Ecal)
    q = s.calibrate(est_cal, err_cal, miss=MISS)
    s.set_offset(q)
    f_te, est_te = infer_all(n_te)
    err = _rel(f_te, E_te)
    guess = _rel(np.broadcast_to(Etr.mean(0, keepdims=True), E_te.shape), E_te)
    accepted = est_te <= THRESHOLD
    violations = float(np.mean(accepted & (err > THRESHOLD)))  # accepted although truly above the threshold
    bound_misses = float(np.mean(err > est_te))                 # the calibrated estimate under the true error

    # inference time per sample at batch 256 against the plain method per sample on the same GPU
    nb = torch.from_numpy(n_te[:min(256, N_TEST)]).to(dev)
    for _ in range(3):
        s.infer(nb)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(20):
        s.infer(nb)
    torch.cuda.synchronize()
    infer_per_sample = (time.perf_counter() - t0) / 20 / len(nb)
    s.close()

    report = {
        "orders": "15x15", "train": n_train, "calibration": n_cal, "held_out": N_TEST, "steps": STEPS, "batch": B,
        "train_s": train_s, "field_loss_first": float(first), "field_loss_last": float(last),
        "held_out_rel_l2": {"median": float(np.median(err)), "p10": float(np.percentile(err, 10)),
                            "p90": float(np.percentile(err, 90)), "max": float(err.max()),
                            "below_5e-2": float(np.mean(err <= THRESHOLD))},
        "mean_field_guess_rel_l2_median": float(np.median(guess)),
        "gate": {"threshold": THRESHOLD, "miss": MISS, "q": float(q), "accepted": float(accepted.mean()),
                 "violations": violations, "estimate_below_true": bound_misses},
        "time_per_sample_s": {"plain_method_gpu": plain_per_sample, "surrogate_inference": infer_per_sample,
                              "speedup": plain_per_sample / infer_per_sample},
        "oracle_check": {"seeds": check_seeds, "oracle_s_per_solve": float(np.mean(oracle_s))},
    }
    print("config5 " + json.dumps(report))
    assert last < 0.2 * first
    assert np.median(err) < 0.75 * np.median(guess)  # the default study is small; see the module docstring
    # split-conformal: P(true error > calibrated estimate) <= MISS, up to finite-sample slack
    assert bound_misses <= MISS + 3 * np.sqrt(MISS * (1 - MISS) / N_TEST) + 1.0 / n_cal
    assert violations <= bound_misses
    assert plain_per_sample / infer_per_sample > 1e3
