"""Oracle runs spread over host processes for the larger GPU parity cases
(test infrastructure).  The pool is started with the spawn method, so it is
safe after the test process has initialised CUDA; each worker runs the
unchanged FP64 oracle on whole replicas."""
import multiprocessing as mp
import os


def _kuramoto_replica(task):
    import oracle
    phi0, omega, D, dt, n0, n1, seed, r, Kconst, meanfield, M = task
    return oracle.kuramoto_run(phi0, omega, D, dt, n0, n1, seed, r, Kconst=Kconst, meanfield=meanfield,
                               sample_every=M)


def kuramoto_replicas(tasks, procs=None):
    """oracle.kuramoto_run for each task tuple (phi0, omega, D, dt, n0, n1,
    seed, replica, Kconst, meanfield, sample_every), in parallel; returns the
    list of (phi, r) in task order."""
    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:
        cores = os.cpu_count() or 1
    procs = max(1, min(procs or cores, len(tasks)))
    if procs == 1:
        return [_kuramoto_replica(t) for t in tasks]
    with mp.get_context("spawn").Pool(procs) as pool:
        return pool.map(_kuramoto_replica, tasks, chunksize=1)
