"""Autotuner: picks launch and schedule parameters by timing real solves.

* ``tune_batch`` -- for a batch: inner cycles per refinement step, nodes per
  work item (the tile) and CTAs per level launch, searched coordinate-wise
  (cycles, then tile, then CTAs), each candidate timed on the caller's batch.
* ``tune_inner_cycles`` -- for one solve in a refinement form: inner cycles
  per outer step.
* ``sweep_refinement`` / ``sweep_batch`` -- time-to-residual over the
  smoother, its sweeps and the inner cycles (the smoother comparison the
  paper makes for the plain form, for the refinement and batched forms).

Timing uses CUDA events on torch's current stream around whole solves from
u = 0 after one untimed solve per candidate (graph capture, first-touch).
"""
from __future__ import annotations


def _time(torch, fn, reps=1):
    fn()  # warm-up: graph capture and first touch
    s = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(s)
    for _ in range(reps):
        fn()
    e1.record(s)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def tune_batch(dims, ns, fd, ud, rtol=1e-10, ks=(2, 4, 6, 8, 10, 12),
               chunks=(512, 1024, 2048, 4096, 8192),
               ctas=(152, 304, 608, 1216, 2432, 4864), **kw):
    """Returns (best parameter dict, list of (params, ms) tried).  Coordinate
    search (inner cycles, then tile, then CTAs), then inner cycles and tile
    once more at the chosen CTA count; settings already timed are reused."""
    import torch
    from .gmg import Batch

    tried = []
    seen = {}

    def measure(p):
        key = (p["inner_cycles"], p["chunk"], p["ctas"])
        if key in seen:
            return seen[key]
        with Batch(dims, ns, inner_cycles=p["inner_cycles"], chunk=p["chunk"], ctas=p["ctas"],
                   **kw) as B:
            def run():
                for u in ud:
                    u.zero_()
                _, _, _, conv = B.solve(fd, ud, rtol)
                assert conv
            ms = _time(torch, run)
        tried.append((dict(p), ms))
        seen[key] = ms
        return ms

    best = {"inner_cycles": ks[0], "chunk": 1024, "ctas": 608}
    for key, values in (("inner_cycles", ks), ("chunk", chunks), ("ctas", ctas),
                        ("inner_cycles", ks), ("chunk", chunks)):
        scores = {}
        for v in values:
            p = dict(best)
            p[key] = v
            scores[v] = measure(p)
        best[key] = min(scores, key=scores.get)
    return best, tried


def tune_inner_cycles(d, n, f, u, precision, ks=(1, 2, 3, 4, 5), rtol=1e-10, **kw):
    """Returns (best k, {k: ms})."""
    import torch
    from .gmg import Solver

    out = {}
    for k in ks:
        with Solver(d, n, precision=precision, inner_cycles=k, **kw) as S:
            def run():
                u.zero_()
                _, _, conv = S.solve(f, u, rtol)
                assert conv
            out[k] = _time(torch, run)
    return min(out, key=out.get), out


def sweep_refinement(d, n, f, u, precision, smoothers, nus, ks=(1, 2, 3, 4), rtol=1e-10,
                     maxit=200):
    """Time-to-rtol of a refinement form over smoother x (nu1 = nu2 = nu) x
    inner cycles.  smoothers: (name, omega) pairs.  Returns rows
    {"smoother", "omega", "nu", "k", "steps", "converged", "ms"} (ms None when
    maxit outer steps did not reach rtol) and the fastest converged row."""
    import torch
    from .gmg import Solver

    rows = []
    for sm, om in smoothers:
        for nu in nus:
            for k in ks:
                with Solver(d, n, precision=precision, inner_cycles=k, smoother=sm, omega=om,
                            nu1=nu, nu2=nu, maxit=maxit) as S:
                    u.zero_()
                    steps, _, conv = S.solve(f, u, rtol)  # also the warm-up

                    def run():
                        u.zero_()
                        S.solve(f, u, rtol)
                    ms = _time(torch, run) if conv else None
                rows.append({"smoother": sm, "omega": om, "nu": nu, "k": k, "steps": steps,
                             "converged": conv, "ms": ms})
    ok = [r for r in rows if r["converged"]]
    return rows, (min(ok, key=lambda r: r["ms"]) if ok else None)


def sweep_batch(dims, ns, fd, ud, precision, smoothers, nus, ks=(1, 2, 3), chunk=0, ctas=0,
                rtol=1e-10, maxit=200):
    """The same for a batch (fixed tile and CTA count): rows
    {"smoother", "omega", "nu", "k", "steps", "converged", "ms"} and the
    fastest converged row."""
    import torch
    from .gmg import Batch

    rows = []
    for sm, om in smoothers:
        for nu in nus:
            for k in ks:
                with Batch(dims, ns, smoother=sm, omega=om, nu1=nu, nu2=nu,
                           precision=precision, inner_cycles=k, chunk=chunk, ctas=ctas,
                           maxit=maxit) as B:
                    for u in ud:
                        u.zero_()
                    _, _, steps, conv = B.solve(fd, ud, rtol)

                    def run():
                        for u in ud:
                            u.zero_()
                        B.solve(fd, ud, rtol)
                    ms = _time(torch, run) if conv else None
                rows.append({"smoother": sm, "omega": om, "nu": nu, "k": k, "steps": steps,
                             "converged": conv, "ms": ms})
    ok = [r for r in rows if r["converged"]]
    return rows, (min(ok, key=lambda r: r["ms"]) if ok else None)
