"""Oracle results shared by the GPU parity tests (computed once per session).

Only oracle/ is called here; nothing comes from the CUDA path."""
import functools
import multiprocessing as mp

import numpy as np

import oracle
import workloads


@functools.lru_cache(maxsize=None)
def uniform_direct(n, seed, kappa):
    """Full direct sum (quadrature reaction kernel) for the uniform workload."""
    x, y, q = workloads.uniform(n, seed=seed)
    u, g = oracle.direct(x, y, q, kappa=kappa)
    return x, y, q, u, g


def _closed_chunk(args):
    xs, ys, qs, idx, kappa = args
    import oracle as o
    return o.direct_closed(xs, ys, qs, idx, kappa)


def sampled_closed(x, y, q, idx, kappa, procs=None):
    """Direct sum at the sampled targets idx (closed-form reaction kernel),
    spread over a spawn process pool."""
    procs = procs or min(16, max(1, mp.cpu_count()))
    chunks = [c for c in np.array_split(np.asarray(idx), procs) if len(c)]
    ctx = mp.get_context("spawn")
    with ctx.Pool(len(chunks)) as pool:
        res = pool.map(_closed_chunk, [(x, y, q, c, kappa) for c in chunks])
    u = np.concatenate([r[0] for r in res])
    g = np.concatenate([r[1] for r in res])
    return u, g


@functools.lru_cache(maxsize=None)
def clustered_sampled(n, seed, kappa):
    """The clustered workload and the oracle at 64 sampled points, half of
    them with y < 0.06 (closed-form reaction kernel)."""
    x, y, q = workloads.clustered(n, seed=seed)
    near = np.flatnonzero(y < 0.06)
    far = np.flatnonzero(y >= 0.06)
    g0 = np.random.Generator(np.random.PCG64(1))
    idx = np.sort(np.concatenate([g0.choice(near, 32, replace=False),
                                  g0.choice(far, 32, replace=False)]))
    u, g = sampled_closed(x, y, q, idx, kappa)
    return x, y, q, idx, u, g
