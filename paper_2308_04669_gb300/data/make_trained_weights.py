"""Writes nedf_thousand_trained.npz: the NeDF weights of the 1024-instance workload's three object
types after the bench's training schedule (per type 2^22 plain-method labels with seed 2 + type, 20,000
Adam steps of 65,536 rays at lr 1e-3, BF16 tensor-core training).  Training steps are deterministic,
so on the same GPU model the bench's own training reproduces these weights bit for bit; the bench's
reference arm (the FP64 oracle) renders with them.

    python paper_2308_04669_gb300/data/make_trained_weights.py [--steps N] [--batch B] [--rays R]
"""
import argparse
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--batch", type=int, default=65536)
    ap.add_argument("--rays", type=int, default=1 << 22)
    ap.add_argument("--out", default=os.path.join(HERE, "nedf_thousand_trained.npz"))
    args = ap.parse_args()
    import torch
    from paper_2308_04669_gb300 import build, scenegen as sg
    build.build()
    from paper_2308_04669_gb300 import native
    sc = sg.thousand_scene()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    r = native.renderer_for(sc, precision=native.PREC_BF16, stream=stream)
    out = {}
    for t in range(len(sc.types)):
        r.make_labels(t, args.rays, 2 + t, 256, 8)
    for t in range(len(sc.types)):
        for _ in range(args.steps):
            r.train_step(t, args.batch, 1e-3)
        out[f"type{t}"] = r.get_nedf_weights(t, sc.types[t].nedf_w.shape[0]).astype(np.float32)
    torch.cuda.synchronize()
    r.close()
    np.savez(args.out, **out, steps=args.steps, batch=args.batch, rays=args.rays)
    print("wrote", args.out)


if __name__ == "__main__":
    main()
