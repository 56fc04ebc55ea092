"""Hyper-parameter sweeps and model-selection quality on synthetic cubes.

The synthetic analogues of the paper's ablations (Sec. IV-E: the split of a
fixed budget of updates between K1, K2 and T; T at K1 = K2 = 5; the ensemble
size M) and of its model-selection illustration (Fig. MSP): every point runs
an ensemble through the library on a seeded synthetic cube with known
endmembers and abundances, times the solve, and scores the runs against the
ground truth with eqs. (RMSE) and (SAD).  Algorithm 2's pick is compared with
the run of lowest RMSE (the one an oracle with the ground truth would pick).

    python -m paper_2209_11002_gb300.sweep --study kkt      # (K1, K2, T) at T (K1 + K2) = 1000
    python -m paper_2209_11002_gb300.sweep --study t        # T at K1 = K2 = 5
    python -m paper_2209_11002_gb300.sweep --study m        # M in {10, 20, 50, 100}
    python -m paper_2209_11002_gb300.sweep --study select   # Algorithm 2 vs the best-RMSE run, several cubes

Each point prints one JSON line.  Needs a CUDA GPU (the solves run in the
library); the scoring is host-side numpy.
"""
from __future__ import annotations

import argparse
import json
import sys
from typing import Dict, List, Sequence

import numpy as np

from paper_2209_11002_gb300 import edaa, metrics, synth

SHAPES = {"jasper": synth.JASPER_ENSEMBLE, "samson": synth.SAMSON_EDAA, "urban": synth.URBAN_PRECISION,
          "apex": synth.APEX_UNROLLED}
PRECISIONS = {"fp32": edaa.FP32, "tf32": edaa.TF32, "bf16": edaa.BF16, "tf32x3": edaa.TF32X3}


def make_cube(shape: str, seed: int, M: int, gammas: Sequence[float]):
    spec = dict(SHAPES[shape])
    spec.update(seed=seed, M=M, gamma_choices=tuple(gammas))
    return synth.make_cube(**{k: v for k, v in spec.items()})


def run_point(cube, T: int, K1: int, K2: int, precision: str = "fp32", repeats: int = 3,
              autotune: int = 1) -> Dict[str, object]:
    """One ensemble solve of `cube` (timed over `repeats` solves after a
    warm-up), Algorithm 2's selection, and every run scored against the
    cube's ground truth."""
    import torch
    X = torch.from_numpy(cube.pixel_major()).cuda()
    stream = torch.cuda.Stream()
    with edaa.Context([dict(X=X, p=cube.p, seeds=cube.seeds, gammas=cube.gammas)], stream=stream, T=T, K1=K1, K2=K2,
                      precision=PRECISIONS[precision], autotune=autotune) as ctx:
        ctx.solve()
        ctx.sync()
        ms = []
        for _ in range(repeats):
            ctx.reset()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.solve()
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        best, fit, mu = ctx.select(0)
        scores = []
        for m in range(cube.M):
            E, A, B = ctx.get(0, m, device="cpu")
            scores.append(metrics.evaluate(cube.E_true, cube.A_true, E, A))
    rmse = [s["rmse"] for s in scores]
    sad = [s["sad"] for s in scores]
    q = metrics.selection_quality(rmse, best)
    run_steps = cube.M * T * (K1 + K2)
    return {"L": cube.L, "N": cube.N, "p": cube.p, "M": cube.M, "T": T, "K1": K1, "K2": K2, "precision": precision,
            "solve_ms": float(np.median(ms)), "run_steps_per_s": run_steps / (float(np.median(ms)) / 1e3),
            "selected": best, "selected_rmse": rmse[best], "selected_sad": sad[best],
            "best_rmse": float(min(rmse)), "best_sad": float(min(sad)), "median_rmse": float(np.median(rmse)),
            "selection": q, "fit_selected": float(fit[best]), "mu_selected": float(mu[best])}


def study_points(study: str) -> List[Dict[str, int]]:
    if study == "kkt":  # a fixed budget of T (K1 + K2) = 1000 updates per run
        return [dict(K1=k, K2=k, T=500 // k) for k in (1, 2, 5, 10, 25, 50)]
    if study == "t":
        return [dict(K1=5, K2=5, T=t) for t in (10, 25, 50, 100, 200)]
    if study == "m":
        return [dict(K1=5, K2=5, T=100, M=m) for m in (10, 20, 50, 100)]
    raise ValueError(study)


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--study", default="kkt", choices=["kkt", "t", "m", "select"])
    ap.add_argument("--shape", default="jasper", choices=sorted(SHAPES))
    ap.add_argument("--precision", default="fp32", choices=sorted(PRECISIONS))
    ap.add_argument("--M", type=int, default=50)
    ap.add_argument("--cubes", type=int, default=5, help="cubes (seeds) of the selection study")
    ap.add_argument("--seed", type=int, default=2000)
    ap.add_argument("--gammas", default="0.5,1,2", help="step factors the runs draw from (eq. eta0A)")
    args = ap.parse_args(argv)
    edaa.load_library()
    gammas = [float(g) for g in args.gammas.split(",")]
    if args.study == "select":
        agg = []
        for c in range(args.cubes):
            cube = make_cube(args.shape, args.seed + c, args.M, gammas)
            r = run_point(cube, 100, 5, 5, args.precision)
            r["cube_seed"] = args.seed + c
            agg.append(r)
            print(json.dumps(r), flush=True)
        print(json.dumps({"study": "select", "cubes": len(agg), "shape": args.shape, "M": args.M,
                          "selected_is_best_fraction": float(np.mean([r["selection"]["selected_is_best"] for r in agg])),
                          "mean_rank": float(np.mean([r["selection"]["rank"] for r in agg])),
                          "mean_regret_rmse": float(np.mean([r["selection"]["regret"] for r in agg])),
                          "mean_selected_rmse": float(np.mean([r["selected_rmse"] for r in agg])),
                          "mean_median_rmse": float(np.mean([r["median_rmse"] for r in agg]))}), flush=True)
        return 0
    for pt in study_points(args.study):
        M = pt.pop("M", args.M)
        cube = make_cube(args.shape, args.seed, M, gammas)
        r = run_point(cube, pt["T"], pt["K1"], pt["K2"], args.precision)
        r["study"] = args.study
        print(json.dumps(r), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
