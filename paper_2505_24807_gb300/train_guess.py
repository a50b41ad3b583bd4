"""Trains the learned Davidson guess/preconditioner network on the GPU and
writes its weights (float32, xs_mlp_nparams() values) to a file.

Training data: seeded molecules of 20-120 atoms (molgen.config_sized, seeds
1000 + s), their ground states and TDHF roots from libxs itself, pair features
and targets from xs_mlp_features / xs_mlp_targets; the network is trained by
libxs's own kernels (xs_mlp_train).  The training record goes to a JSON file
beside the weights (same name, .json).

  python -m paper_2505_24807_gb300.train_guess --molecules 4096 --epochs 20 --out guess_weights.f32
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import molgen  # noqa: E402
from paper_2505_24807_gb300 import xs  # noqa: E402


def train(n_mol=256, nroots=8, pairs=2048, epochs=60, seed=1, ctx=None):
    params = molgen.make_params(0)
    own = ctx is None
    if own:
        ctx = xs.xs_create(0)
        xs.xs_set_params(ctx, molgen.params_table(params))
    mols = [molgen.config_sized(1000 + s, 20 + (s * 7919) % 101) for s in range(n_mol)]
    t0 = time.perf_counter()
    xs.xs_ground_state(ctx, mols)
    xs.xs_excited(ctx, method=xs.XS_TDHF, nroots=nroots, tol=1e-6, batched=1, n_mol=len(mols))
    feats, targs = [], []
    for i in range(len(mols)):
        F, pr = xs.xs_mlp_features(ctx, i, pairs)
        feats.append(F)
        targs.append(xs.xs_mlp_targets(ctx, i, pr))
    F = np.concatenate(feats)
    T = np.concatenate(targs)
    perm = np.random.default_rng(seed).permutation(len(F))
    xs.xs_mlp_init(ctx, seed=seed)
    loss = xs.xs_mlp_train(ctx, F[perm], T[perm], epochs=epochs, batch=4096, lr=2e-3)
    w = xs.xs_mlp_get_weights(ctx)
    info = dict(molecules=n_mol, atoms="20-120", molecule_seeds=f"1000..{1000 + n_mol - 1}", nroots=nroots,
                pairs_per_molecule=pairs, samples=int(len(F)), epochs=epochs, loss_first=float(loss[0]),
                loss_last=float(loss[-1]), seconds=time.perf_counter() - t0)
    if own:
        xs.xs_destroy(ctx)
    return w, info


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--molecules", type=int, default=256)
    ap.add_argument("--epochs", type=int, default=60)
    ap.add_argument("--out", required=True)
    args = ap.parse_args()
    w, info = train(args.molecules, epochs=args.epochs)
    w.astype(np.float32).tofile(args.out)
    with open(os.path.splitext(args.out)[0] + ".json", "w") as f:
        json.dump(info, f, indent=1)
    print(json.dumps(info))


if __name__ == "__main__":
    main()
