"""Calibrate the server's admission model (gd_query_footprint) on a mesh pool.

The server admits requests by their predicted work-buffer bytes: 16 B per
entry of the two fronts at the largest level and of the leaf pairs, 72 B per
float64 candidate, each count a power law c * s^p in s = sqrt(T_A) +
sqrt(T_B).  This script measures those counts on single queries (gd_stats
after gd_min_distance / gd_max_distance) for random pairs and placements of
a pool of meshes, and prints p (least squares in log-log) and c (the chosen
quantile of the residuals, so that that fraction of the measured queries lies
below each curve).  The constants in csrc/gd_serve.cu came from

    python -m paper_2411_11244_gb300.fit_footprint --requests 800 --quantile 0.99

on one GB300 with the 64-mesh pool of synth.mesh_pool (seed 0): front
349 s^1.223, leaf pairs 71.5 s^1.514, candidates 570 s^0.642.  Needs a GPU.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import sys


def collect(n_requests: int, seed: int = 7, pool_seed: int = 0):
    import numpy as np
    from paper_2411_11244_gb300 import build, gdist as G, synth
    build.build()
    ctx = G.gd_ctx_create(0)
    pool = synth.mesh_pool(64, seed=pool_seed)
    hs, rad, nt = [], [], []
    for m in pool:
        h = G.gd_mesh_create(ctx, *m)
        G.gd_bvh_build(h, ctx=ctx)
        hs.append(h)
        rad.append(float(np.max(np.linalg.norm(m[0].astype(np.float64), axis=1))))
        nt.append(len(m[1]))
    rng = np.random.default_rng(seed)
    rows = []
    for i in range(n_requests):
        a, b = int(rng.integers(0, 64)), int(rng.integers(0, 64))
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        xb = synth.xform(synth.random_rotation(rng), d * rng.uniform(0.5, 1.5) * (rad[a] + rad[b]))
        fn = G.gd_min_distance if i % 4 else G.gd_max_distance
        fn(ctx, hs[a], hs[b], synth.identity_xform(), xb)
        st = G.gd_get_stats(ctx)
        rows.append({"ta": nt[a], "tb": nt[b], "front_max": max(st["front"]), "leaf_pairs": st["leaf_pairs"],
                     "candidates": st["candidates"]})
    for h in hs:
        G.gd_mesh_destroy(h)
    G.gd_ctx_destroy(ctx)
    return rows


def fit(rows, quantile: float = 0.99):
    import numpy as np
    s = np.array([math.sqrt(r["ta"]) + math.sqrt(r["tb"]) for r in rows])
    out = {}
    for key in ("front_max", "leaf_pairs", "candidates"):
        y = np.array([max(1, r[key]) for r in rows], dtype=float)
        p, _ = np.polyfit(np.log(s), np.log(y), 1)
        c = math.exp(float(np.quantile(np.log(y) - p * np.log(s), quantile)))
        out[key] = {"c": c, "p": float(p)}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--requests", type=int, default=800)
    ap.add_argument("--quantile", type=float, default=0.99)
    ap.add_argument("--rows", help="write the measured rows (JSON) here")
    args = ap.parse_args()
    rows = collect(args.requests)
    if args.rows:
        json.dump(rows, open(args.rows, "w"))
    print(json.dumps(fit(rows, args.quantile), indent=1))


if __name__ == "__main__":
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    main()
