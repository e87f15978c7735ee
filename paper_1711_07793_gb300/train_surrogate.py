"""Train the learned penumbra surrogate on the GPU and write a checkpoint.

    python -m paper_1711_07793_gb300.train_surrogate [--samples 16777216] [--out PATH]

Training data: every edge fragment (filtering mode) of seeded 4096^2 /
3840x2160 scenes (the C4 recipe of rbsm_scenes, seeds 0, 1, 2, ...) with its
exact RSMSS answer, until `--samples` are collected.  Training: Adam on
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


def collect(samples_wanted, first_seed=0, log=print):
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
        N.check("rbsm_mlp_dataset", N.lib().rbsm_mlp_dataset(
            ctypes.byref(m), ctypes.byref(fr), ctypes.byref(p), ctypes.c_void_p(samples.data_ptr()),
            samples_wanted, ctypes.c_void_p(counter.data_ptr()), _stream_handle(None)))
        count = min(int(counter.item()), samples_wanted)
        seeds.append(seed)
        log("seed %d: %d samples" % (seed, count))
        seed += 1
    return samples, count, seeds


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--samples", type=int, default=1 << 24)
    ap.add_argument("--epochs", type=int, default=6)
    ap.add_argument("--batch", type=int, default=8192)
    ap.add_argument("--lr", type=float, default=3e-3)
    ap.add_argument("--init-seed", type=int, default=0)
    ap.add_argument("--out", default=DEFAULT_CHECKPOINT)
    args = ap.parse_args(argv)

    sys.path.insert(0, ROOT)
    from . import build as lib_build
    lib_build.build()
    import rbsm_scenes as sc
    from .surrogate import Surrogate

    t0 = time.time()
    samples, count, seeds = collect(args.samples, log=lambda m: print(m, file=sys.stderr))
    t_data = time.time() - t0
    net = Surrogate(sc.mlp_init(args.init_seed))
    torch.cuda.synchronize()
    t1 = time.time()
    hist = net.train(samples, count, epochs=args.epochs, batch=args.batch, lr=args.lr, seed=args.init_seed,
                     log=lambda m: print(m, file=sys.stderr))
    torch.cuda.synchronize()
    t_train = time.time() - t1
    os.makedirs(os.path.dirname(os.path.abspath(args.out)), exist_ok=True)
    meta = {"data": "edge fragments of rbsm_scenes.config4 seeds %d..%d (4096^2 map, 3840x2160)"
                    % (seeds[0], seeds[-1]),
            "samples": count, "epochs": args.epochs, "batch": args.batch, "lr": args.lr,
            "init_seed": args.init_seed, "loss_per_epoch": hist,
            "device": torch.cuda.get_device_name(0)}
    net.save(args.out, meta)
    report = dict(meta, data_seconds=round(t_data, 2), train_seconds=round(t_train, 2),
                  steps=net.step, checkpoint=os.path.relpath(args.out, ROOT))
    print(json.dumps(report))


if __name__ == "__main__":
    main()
