"""Train the two-drop surrogate on solver trajectories and evaluate it.

    python -m paper_2011_00814_gb300.train_surrogate --out weights.npz [--json summary.json]

Steps: seeded two-drop cases (``inputs.two_drops``) -> trajectories of the
batched FP32 solver, one snapshot every K steps -> normalisation statistics
-> Adam on the library's BF16 network kernels -> on held-out cases, the
one-call phase-field error of the network and of the persistence map, and
the controller's time-to-solution against the plain solver over ``calls``
calls.  Writes the weights (FP32, with the normalisation) and a JSON summary.

The controller's check tolerance is then calibrated on ``--calibrate``
further held-out problems (seeds after the evaluated ones) and written next
to the weights (``surrogate.calibration_path``).  With ``--weights`` an
existing weights file is calibrated without training:

    python -m paper_2011_00814_gb300.train_surrogate \
        --weights paper_2011_00814_gb300/data/unet_two_drops_256.npz --calibrate 8
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np

from . import build, gpe2p, inputs
from . import surrogate as S


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--K", type=int, default=64)
    ap.add_argument("--train", type=int, default=64, help="training trajectories")
    ap.add_argument("--test", type=int, default=8, help="held-out trajectories")
    ap.add_argument("--snapshots", type=int, default=12)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--levels", type=int, default=S.LEVELS)
    ap.add_argument("--channels", type=str, default=",".join(str(c) for c in S.CHANNELS))
    ap.add_argument("--calls", type=int, default=64, help="controller calls of the time-to-solution runs")
    ap.add_argument("--compare", type=int, default=2, help="held-out cases in the time-to-solution runs")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--out", type=str, default="")
    ap.add_argument("--json", type=str, default="")
    ap.add_argument("--weights", type=str, default="", help="calibrate these weights instead of training")
    ap.add_argument("--calibrate", type=int, default=8, help="held-out problems of the tolerance calibration")
    ap.add_argument("--skip-eval", type=int, default=4,
                    help="held-out problems kept for evaluation (the benchmark's), skipped by the calibration")
    a = ap.parse_args(argv)
    import torch
    build.build()
    gpe2p.lib()
    chans = tuple(int(c) for c in a.channels.split(","))
    summary = {"args": vars(a)}
    if a.weights:
        sur = S.Surrogate.load(a.weights, max_batch=a.batch)
        calibrate(sur, a, a.weights)
        sur.close()
        return
    if not a.out:
        ap.error("--out is required when training")

    train_cases = [inputs.two_drops(a.seed * 100000 + s, n=a.n) for s in range(a.train)]
    test_cases = [inputs.two_drops(a.seed * 100000 + 50000 + s, n=a.n) for s in range(a.test)]
    D, t_gen = S.generate(train_cases, a.snapshots, a.K, group=256)
    Dt, t_gen_t = S.generate(test_cases, a.snapshots, a.K, group=256)
    steps_gen = (a.train + a.test) * a.snapshots * a.K
    summary["generate"] = {"seconds": t_gen + t_gen_t, "instance_steps": steps_gen,
                           "cell_updates_per_s": steps_gen * a.n * a.n / (t_gen + t_gen_t),
                           "dataset_gb": D.numel() * 4 / 1e9}
    print(json.dumps(summary["generate"]), flush=True)

    sur = S.Surrogate(n=a.n, K=a.K, levels=a.levels, channels=chans, max_batch=a.batch, seed=a.seed + 1)
    mean, scale, oscale = S.dataset_stats(D)
    sur.set_stats(mean, scale, oscale)
    summary["normalisation"] = {"in_mean": mean.tolist(), "in_scale": scale.tolist(), "out_scale": oscale.tolist()}
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hist = S.train(sur, D, a.steps, batch=a.batch, lr=a.lr, seed=a.seed, log_every=max(a.steps // 20, 1))
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    fl = 3.0 * sur.flops(a.batch) * a.steps
    summary["train"] = {"seconds": t_train, "steps": a.steps, "batch": a.batch, "loss": hist,
                        "params": sur.net.nparam, "forward_gflop_per_sample": sur.flops(1) / 1e9,
                        "approx_tflops": fl / t_train / 1e12}
    print(json.dumps({k: v for k, v in summary["train"].items() if k != "loss"}), "loss", hist[0], hist[-1],
          flush=True)

    pairs = [(t, k) for t in range(a.test) for k in range(a.snapshots)]
    errs = S.one_call_errors(sur, Dt, pairs)
    ne = np.array([e for e, _ in errs])
    pe = np.array([e for _, e in errs])
    summary["held_out_one_call"] = {"pairs": len(pairs), "net_mean": float(ne.mean()), "net_max": float(ne.max()),
                                    "persistence_mean": float(pe.mean()), "persistence_max": float(pe.max()),
                                    "frac_under_tol": float(np.mean(ne <= 2e-2))}
    print(json.dumps(summary["held_out_one_call"]), flush=True)
    del D
    torch.cuda.empty_cache()

    runs = []
    for c in range(min(a.compare, a.test)):
        torch.cuda.synchronize()
        prm, f = test_cases[c]
        for pers in (False, True):
            r = S.compare_to_solver(sur, prm, f, calls=a.calls, repeats=2, persistence=pers)
            r["case"] = c
            r["r_rho"] = prm["r_rho"]
            r["surrogate"] = "persistence" if pers else "network"
            r["stats"].pop("check_l2", None)
            runs.append(r)
            print(json.dumps(r), flush=True)
    summary["time_to_solution"] = runs
    sur.save(a.out, meta={"K": a.K, "train": a.train, "snapshots": a.snapshots, "steps": a.steps,
                          "seed": a.seed})
    summary["calibration"] = calibrate(sur, a, a.out)
    if a.json:
        with open(a.json, "w") as fh:
            json.dump(summary, fh, indent=1)
    sur.close()


def calibrate(sur, a, weights_path):
    """Calibrate the check tolerance on held-out problems and write it beside the weights."""
    n = sur.n
    first = a.seed * 100000 + 50000 + a.skip_eval
    cases = [inputs.two_drops(first + c, n=n) for c in range(a.calibrate)]
    cal = S.calibrate_tolerance(sur, cases, calls=a.calls)
    cal["seeds"] = [first, first + a.calibrate - 1]
    cal["weights"] = os.path.basename(weights_path)
    with open(S.calibration_path(weights_path), "w") as fh:
        json.dump(cal, fh, indent=1)
    print(json.dumps(cal), flush=True)
    return cal


if __name__ == "__main__":
    main()
