"""Oracle runs for a spawned process pool (test infrastructure).

The workers import only numpy and the oracle, never torch or CUDA: the pool is started with
the "spawn" method, so that no child inherits a CUDA context from the test process."""
import concurrent.futures as cf
import multiprocessing as mp
import os

import numpy as np


def _run_1d(args):
    """(n, dx, bc, U0 [3][1][n], T) -> (U_T, steps): CFL steps clipped at T."""
    from oracle import oracle as O
    n, dx, bc, U0, T = args
    P = O.problem(O.EULER1D, n, 1, dx=dx, bc_x=bc)
    return O.run(P, U0, T)


def _set_threads(n):
    from oracle import oracle as O
    O.set_num_threads(n)


def pool(workers: int | None = None, threads: int = 1) -> cf.ProcessPoolExecutor:
    """A spawned pool; each worker runs the oracle on `threads` OpenMP threads."""
    workers = workers or max(1, min(32, os.cpu_count() or 1))
    return cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn"),
                                  initializer=_set_threads, initargs=(threads,))


def run_1d_many(jobs, workers: int | None = None, threads: int = 1):
    """The 1D Euler runs `jobs` (tuples as _run_1d takes them) on a spawned pool, in order."""
    with pool(workers, threads) as ex:
        return list(ex.map(_run_1d, jobs))


def one_ulp(U: np.ndarray, draw: int) -> np.ndarray:
    """U with every entry moved by one unit in the last place (relative 2^-52), signs seeded."""
    sign = np.random.default_rng(1000 + draw).choice([-1.0, 1.0], size=U.shape)
    return U * (1.0 + 2.0 ** -52 * sign)
