"""Train the warm-start network (8 raw channels + the upsampled coarse solution) on volumes
labelled by the plain power iteration and save its parameters
(paper_2212_08058_gb300/data/warmstart_c8_coarse.npy).

    python -m paper_2212_08058_gb300.train_warmstart [--volumes 2000] [--epochs 3]

Prints one JSON line with the hold-out cosine loss before and after training.
"""
from __future__ import annotations

import argparse
import json

from . import build, sfseg, warmstart


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--volumes", type=int, default=2000)
    ap.add_argument("--holdout", type=int, default=100)
    ap.add_argument("--epochs", type=int, default=3)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--out", default=warmstart.DEFAULT_WEIGHTS)
    args = ap.parse_args()
    build.build()
    net = sfseg.WarmStartNet(9, seed=args.seed)
    stats = warmstart.train(net, n_train=args.volumes, n_holdout=args.holdout, epochs=args.epochs, lr=args.lr,
                            log=lambda m: None)
    warmstart.save(net, args.out)
    stats["weights"] = args.out
    print(json.dumps(stats))


if __name__ == "__main__":
    main()
