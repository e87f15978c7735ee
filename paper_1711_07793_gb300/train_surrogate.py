"""Train the learned penumbra surrogate on the GPU and write a checkpoint.

    python -m paper_1711_07793_gb300.train_surrogate [--samples 16777216] [--out PATH]

Training data: the edge fragments (filtering mode) of seeded 4096^2 /
3840x2160 scenes (the C4 recipe of rbsm_scenes, seeds 0, 1, 2, ...) whose
Listing 3 walks stop inside the 5x5 window the network sees (the only ones
the batch's guard lets it answer; --all-edges keeps every edge fragment),
with their exact RSMSS answers, until `--samples` are collected.
Calibration: the trained network answers the edge fragments of the scenes
that follow (--cal-samples of them); the 5x5 patterns on which it stayed
within --trust-error of the exact answer, seen at least --trust-min-count
times, form the trusted-pattern bitmap stored with the checkpoint.  Training: Adam on
shuffled minibatches with a halving learning rate, all in the library's
kernels.  Writes the checkpoint (float32 parameters plus a JSON header with
the dimensions, step count, data recipe and per-epoch losses) and prints a
JSON report line.
"""
import argparse
import json
import os
import sys
import time

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
DEFAULT_CHECKPOINT = os.path.join(HERE, "weights", "surrogate_c4.npz")


def collect(samples_wanted, first_seed=0, log=print, in_window=True):
    import rbsm_scenes as sc
    from .surrogate import SAMPLE_BYTES, Surrogate
    from . import _native as N
    import ctypes
    from .api import frags_desc, map_desc, _params, _stream_handle

    dev = torch.device("cuda")
    samples = torch.empty(samples_wanted * SAMPLE_BYTES, dtype=torch.uint8, device=dev)
    counter = torch.zeros(1, dtype=torch.int64, device=dev)
    seeds = []
    seed = first_seed
    count = 0
    while count < samples_wanted:
        f = sc.config4(seed)
        depth = torch.from_numpy(f.depth).to(dev)
        x, y, z = (torch.from_numpy(a).to(dev) for a in (f.x, f.y, f.z))
        m, fr, p = map_desc(depth), frags_desc(x, y, z), _params(16)
        p.flags = N.RBSM_DATASET_IN_WINDOW if in_window else 0
        N.check("rbsm_mlp_dataset", N.lib().rbsm_mlp_dataset(
            ctypes.byref(m), ctypes.byref(fr), ctypes.byref(p), ctypes.c_void_p(samples.data_ptr()),
            samples_wanted, ctypes.c_void_p(counter.data_ptr()), _stream_handle(None)))
        count = min(int(counter.item()), samples_wanted)
        seeds.append(seed)
        log("seed %d: %d samples" % (seed, count))
        seed += 1
    return samples, count, seeds


def calibrate(net, args, first_seed, in_window=True, log=lambda m: print(m, file=sys.stderr)):
    """Trusted-pattern bitmap: the network answers (the library's tcgen05
    forward pass) the edge fragments of calibration scenes that training did
    not see; a 5x5 pattern is trusted when it occurs at least
    --trust-min-count times there and the largest error of the clamped
    answer against the exact one is at most --trust-error.  Installs the
    bitmap in the network and returns a summary."""
    from .surrogate import Surrogate
    samples, count, seeds = collect(args.cal_samples, first_seed=first_seed, log=log, in_window=in_window)
    out = net.forward(samples, count).cpu().numpy().astype(np.float64)
    rec = Surrogate.unpack(samples, count)
    err = np.abs(np.clip(out[:, 0], 0.0, 1.0) - rec["label"].astype(np.float64))
    order = np.argsort(rec["bits"], kind="stable")
    bits, err = rec["bits"][order], err[order]
    starts = np.flatnonzero(np.r_[True, bits[1:] != bits[:-1]])
    counts = np.diff(np.r_[starts, bits.size])
    worst = np.maximum.reduceat(err, starts)
    trusted = (counts >= args.trust_min_count) & (worst <= args.trust_error)
    net.set_trust(Surrogate.trust_bitmap(bits[starts][trusted]))
    summary = {"seeds": [seeds[0], seeds[-1]], "samples": int(count), "patterns": int(starts.size),
               "trusted_patterns": int(trusted.sum()), "trusted_sample_frac": float(counts[trusted].sum() / count),
               "trust_error": args.trust_error, "trust_min_count": args.trust_min_count}
    log("calibration: %s" % json.dumps(summary))
    return summary


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--samples", type=int, default=1 << 24)
    ap.add_argument("--epochs", type=int, default=6)
    ap.add_argument("--batch", type=int, default=8192)
    ap.add_argument("--lr", type=float, default=3e-3)
    ap.add_argument("--init-seed", type=int, default=0)
    ap.add_argument("--out", default=DEFAULT_CHECKPOINT)
    ap.add_argument("--all-edges", action="store_true",
                    help="train on every edge fragment, not only those whose walks stop inside the window")
    ap.add_argument("--cal-samples", type=int, default=1 << 24,
                    help="calibration samples (scenes after the training ones); 0 = no trusted-pattern bitmap")
    ap.add_argument("--trust-error", type=float, default=0.05,
                    help="a pattern is trusted when the network's largest calibration error on it is at most this")
    ap.add_argument("--trust-min-count", type=int, default=8,
                    help="... and it occurred at least this often in the calibration scenes")
    args = ap.parse_args(argv)

    sys.path.insert(0, ROOT)
    from . import build as lib_build
    lib_build.build()
    import rbsm_scenes as sc
    from .surrogate import Surrogate

    t0 = time.time()
    samples, count, seeds = collect(args.samples, log=lambda m: print(m, file=sys.stderr),
                                    in_window=not args.all_edges)
    t_data = time.time() - t0
    net = Surrogate(sc.mlp_init(args.init_seed))
    torch.cuda.synchronize()
    t1 = time.time()
    hist = net.train(samples, count, epochs=args.epochs, batch=args.batch, lr=args.lr, seed=args.init_seed,
                     log=lambda m: print(m, file=sys.stderr))
    torch.cuda.synchronize()
    t_train = time.time() - t1
    cal = None
    if args.cal_samples > 0:
        cal = calibrate(net, args, first_seed=seeds[-1] + 1, in_window=not args.all_edges)
    os.makedirs(os.path.dirname(os.path.abspath(args.out)), exist_ok=True)
    meta = {"data": "%s of rbsm_scenes.config4 seeds %d..%d (4096^2 map, 3840x2160)"
                    % ("edge fragments" if args.all_edges else "edge fragments whose walks stop inside the 5x5 window",
                       seeds[0], seeds[-1]),
            "in_window": not args.all_edges,
            "samples": count, "epochs": args.epochs, "batch": args.batch, "lr": args.lr,
            "init_seed": args.init_seed, "loss_per_epoch": hist,
            "device": torch.cuda.get_device_name(0), "calibration": cal}
    net.save(args.out, meta)
    report = dict(meta, data_seconds=round(t_data, 2), train_seconds=round(t_train, 2),
                  steps=net.step, checkpoint=os.path.relpath(args.out, ROOT))
    print(json.dumps(report))


if __name__ == "__main__":
    main()
