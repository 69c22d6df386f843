"""Parallel oracle runs for the GPU tests (test infrastructure).

The FP64 oracle solves the cells of a sub-batch independently from the same
state (Section 5.1: the cells of one batch do not interact), so the tests hand
them to a pool of worker processes.  The pool is started with ``spawn`` (a
process forked after the parent has created a CUDA context can hang); every
worker receives the oracle state once, through the pool initialiser, and runs
``oracle.domdec.solve_cell`` unchanged.
"""
from __future__ import annotations

import multiprocessing as mp
import os

from oracle import domdec as odd

_STATE = None


def _init(st):
    global _STATE
    _STATE = st


def _solve(args):
    cell, prob, err, maxit = args
    return odd.solve_cell(_STATE, cell, prob, err=err, maxit=maxit)


def solve_cells(st, jobs, err, maxit, workers=None):
    """[solve_cell(st, cell, prob, err, maxit) for (cell, prob) in jobs], in order."""
    if not jobs:
        return []
    n = workers or min(len(jobs), max(1, (os.cpu_count() or 1)))
    if n <= 1:
        return [odd.solve_cell(st, c, p, err=err, maxit=maxit) for c, p in jobs]
    ctx = mp.get_context("spawn")
    with ctx.Pool(n, initializer=_init, initargs=(st,)) as pool:
        return pool.map(_solve, [(c, p, err, maxit) for c, p in jobs], chunksize=1)


def _trajectory(args):
    import copy

    from paper_2410_08859_gb300 import inputs
    N, s, seed, eps, lam, sweeps = args
    mu, nu = inputs.mixture_small(N=N, seed=seed)
    st = odd.init_product(odd.Geometry(N, s), mu.ravel(), nu.ravel(), eps, lam)
    out = []
    for k in range(sweeps):
        log = odd.sweep(st, "AB"[k % 2], "staggered")
        out.append((log, copy.deepcopy(st)))
    return out


def mixture_trajectories(specs, sweeps):
    """Oracle runs (pi0 = mu x nu, staggered, default tolerances) of independent
    problems (N, s, eps, lam, seed), sweeps[j] sweeps of problem j, one worker
    process each: per problem the decision log and the state after every sweep."""
    jobs = [(N, s, seed, eps, lam, k) for (N, s, eps, lam, seed), k in zip(specs, sweeps)]
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(len(jobs), max(1, os.cpu_count() or 1))) as pool:
        return pool.map(_trajectory, jobs, chunksize=1)
