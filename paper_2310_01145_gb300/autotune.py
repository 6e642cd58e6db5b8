"""Autotuner for the solver's launch shape: kernel layout variant x chain length.

For a problem shape (ODE family, d, q, N, dtype) it times fixed-iteration solves for every
compiled layout variant (0: one state row per lane, 1: two rows per lane) and a range of chain
lengths, and records the fastest in a JSON table keyed by the shape.  ``lookup`` returns the
tuned (variant, chain_len) for a problem, falling back to the nearest tuned N of the same
(family, d, q, dtype), else the library defaults (0, 0).

    python -m paper_2310_01145_gb300.autotune --family fitzhugh_nagumo --q 3 --N 1048576
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time

TABLE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning.json")


def _key(kind: int, d: int, q: int, dtype: str, N: int) -> str:
    return f"{kind}:{d}:{q}:{dtype}:{N}"


def load_table(path: str = TABLE) -> dict:
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def lookup(problem, dtype: str, path: str = TABLE):
    """Tuned (variant, chain_len) for a workloads.Problem, or (0, 0)."""
    tab = load_table(path)
    exact = tab.get(_key(problem.kind, problem.d, problem.q, dtype, problem.N))
    if exact:
        return exact["variant"], exact["chain_len"]
    best = None
    for k, v in tab.items():
        kind, d, q, dt, N = k.split(":")
        if (int(kind), int(d), int(q), dt) == (problem.kind, problem.d, problem.q, dtype):
            dist = abs(math.log(int(N)) - math.log(problem.N))
            if best is None or dist < best[0]:
                best = (dist, v)
    if best is None:
        return 0, 0
    v = best[1]
    return v["variant"], 0


def sweep(problem, dtype: str = "f32", iters: int = 6, variants=(0, 1),
          chain_lens=(0, 16, 24, 32, 48, 64, 96, 128), repeats: int = 3):
    import torch
    import paper_2310_01145_gb300 as pit

    tdt = torch.float32 if dtype == "f32" else torch.float64
    ode = pit.ode_from_problem(problem)
    results = []
    for v in variants:
        for L in chain_lens:
            opts = pit.make_opts(dtype=tdt, fixed_iters=iters, want_cov=False, chain_len=L,
                                 variant=v)
            try:
                pit.pit_solve(ode, problem.y0, problem.t0, problem.t1, problem.N, problem.q,
                              opts)
            except pit.PitError as exc:
                results.append({"variant": v, "chain_len": L, "ms": None, "error": str(exc)})
                continue
            torch.cuda.synchronize()
            times = []
            for _ in range(repeats):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                pit.pit_solve(ode, problem.y0, problem.t0, problem.t1, problem.N, problem.q,
                              opts)
                e1.record()
                torch.cuda.synchronize()
                times.append(e0.elapsed_time(e1))
            results.append({"variant": v, "chain_len": L, "ms": min(times) / iters})
    return results


def tune(problem, dtype: str = "f32", path: str = TABLE, **kw) -> dict:
    res = sweep(problem, dtype, **kw)
    ok = [r for r in res if r["ms"] is not None]
    best = min(ok, key=lambda r: r["ms"])
    tab = load_table(path)
    tab[_key(problem.kind, problem.d, problem.q, dtype, problem.N)] = {
        "variant": best["variant"], "chain_len": best["chain_len"],
        "ms_per_iteration": best["ms"], "sweep": res,
        "when": time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime())}
    with open(path, "w") as fh:
        json.dump(tab, fh, indent=1, sort_keys=True)
    return best


def main():
    import workloads as W
    ap = argparse.ArgumentParser()
    ap.add_argument("--family", default="fitzhugh_nagumo")
    ap.add_argument("--q", type=int, default=3)
    ap.add_argument("--N", type=int, nargs="+", default=[2 ** 20])
    ap.add_argument("--dtype", default="f32")
    ap.add_argument("--iters", type=int, default=6)
    ap.add_argument("--out", default=TABLE, help="tuning table to update (JSON)")
    ap.add_argument("--chain-lens", type=int, nargs="+",
                    default=[0, 16, 24, 32, 48, 64, 96, 128])
    args = ap.parse_args()
    make = {"fitzhugh_nagumo": W.fitzhugh_nagumo, "logistic": W.logistic,
            "van_der_pol": W.van_der_pol, "rigid_body": W.rigid_body,
            "lotka_volterra": lambda N, q: W.lotka_volterra(N=N, q=q)}[args.family]
    for N in args.N:
        p = make(N=N, q=args.q)
        best = tune(p, args.dtype, path=args.out, iters=args.iters,
                    chain_lens=tuple(args.chain_lens))
        print(json.dumps({"family": args.family, "q": args.q, "N": N, "dtype": args.dtype,
                          **best}))


if __name__ == "__main__":
    main()
