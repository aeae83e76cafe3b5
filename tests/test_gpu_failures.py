"""Failure detection on the GPU without a GPU fault.

- Bounded device waits: the tensor-core GEMMs (the TMA producers, the MMA
  issuers, the stream-K heads' polls of their partial sums' flags)
  and the Kuramoto mean field with the asynchronous cluster exchange wait on
  mbarriers with a limit of the GPU's nanosecond timer.  A limit of 1 ns makes
  those waits expire on purpose: the kernels drain what they issued, latch
  SDE_ERR_TIMEOUT, and the context stays usable -- after the default limit is
  restored the same context reproduces a fresh context's run bit for bit.
- Allocation failures: sde_debug_fail_allocation makes the nth allocation of
  the next create call fail; every n reports SDE_ERR_NO_MEMORY with a NULL
  context, and a normal create afterwards works.
"""
import numpy as np
import pytest
import torch

from gpu_util import ensure_built, kur_run
from paper_0903_3852_gb300 import inputs, sde

pytestmark = pytest.mark.gpu


def _general(N, R, seed, flags=0):
    ensure_built()
    return sde.Ensemble.kuramoto(sde.SDE_KURAMOTO_GENERAL, N, R, 0.0, 0.02, 0.005, seed, sample_every=10,
                                 flags=flags)


# one-CTA GEMM, CTA-pair GEMM, stream-K GEMM (its heads' flag polls expire too)
@pytest.mark.parametrize("N,R,cluster", [(512, 64, 1), (1024, 128, 2), (2048, 128, 0)])
def test_tensor_core_gemm_wait_expiry_is_reported_and_recovered(N, R, cluster):
    steps = 20
    flags = sde.SDE_FLAG_GEMM_STREAM_K if cluster == 0 else 0
    w = inputs.kuramoto_general(n_osc=N, replicas=R, seed=31)
    K = torch.from_numpy(w["Kmat"]).cuda()
    ref = _general(N, R, 3, flags)
    ref.set_coupling(K)
    phi_ref, r_ref, _ = kur_run(ref, w["phi0"], w["omega"], 0, steps)
    ens = _general(N, R, 3, flags)
    assert ens.tuning()[2] == cluster
    ens.set_coupling(K)
    ens.set_wait_limit(1)
    with pytest.raises(sde.SDEError) as e:
        kur_run(ens, w["phi0"], w["omega"], 0, steps)
    assert e.value.status == sde.SDE_ERR_TIMEOUT
    ens.set_wait_limit(0)
    phi, r, _ = kur_run(ens, w["phi0"], w["omega"], 0, steps)
    assert np.array_equal(phi, phi_ref) and np.array_equal(r, r_ref)


def test_async_meanfield_wait_expiry_is_reported_and_recovered():
    N, R, steps = 4096, 2, 200
    w = inputs.kuramoto_uniform(n_osc=N, replicas=R, seed=32)
    ensure_built()
    kw = dict(sample_every=50, block_threads=512, cluster_ctas=2, flags=sde.SDE_FLAG_ASYNC_EXCHANGE)
    ref = sde.Ensemble.kuramoto(sde.SDE_KURAMOTO_MEANFIELD, N, R, 2.0, 0.05, 0.01, 4, **kw)
    phi_ref, r_ref, _ = kur_run(ref, w["phi0"], w["omega"], 0, steps)
    ens = sde.Ensemble.kuramoto(sde.SDE_KURAMOTO_MEANFIELD, N, R, 2.0, 0.05, 0.01, 4, **kw)
    assert ens.tuning()[2] == 2
    ens.set_wait_limit(1)
    with pytest.raises(sde.SDEError) as e:
        kur_run(ens, w["phi0"], w["omega"], 0, steps)
    assert e.value.status == sde.SDE_ERR_TIMEOUT
    ens.set_wait_limit(0)
    phi, r, _ = kur_run(ens, w["phi0"], w["omega"], 0, steps)
    assert np.array_equal(phi, phi_ref) and np.array_equal(r, r_ref)


@pytest.mark.parametrize("kind", ["josephson", "kuramoto_general", "mlp"])
def test_every_injected_allocation_failure_reports_no_memory(kind):
    ensure_built()
    pt = dict(gamma=0.9, a=4.2, omega=4.9, f=0.1, D=1e-3)

    def create():
        if kind == "josephson":
            return sde.Ensemble.josephson([pt, pt], [100, 50], [300, 200], 0)  # autotuned: scratch too
        if kind == "kuramoto_general":
            return _general(512, 64, 1)
        return sde.Mlp(max_batch=256)

    failures = 0
    for nth in range(1, 64):
        sde.debug_fail_allocation(nth)
        try:
            obj = create()
        except sde.SDEError as e:
            assert e.status == sde.SDE_ERR_NO_MEMORY, str(e)
            failures += 1
            continue
        obj.close()  # nth beyond the call's allocations: nothing failed
        break
    else:
        pytest.fail("create made more than 63 allocations")
    assert failures >= 5
    # disarmed: a normal create and run work
    if kind == "josephson":
        ens = create()
        wj = inputs.josephson_custom([pt, pt], [100, 50], [300, 200], seed=0)
        x = torch.from_numpy(wj["x0"]).cuda()
        v = torch.from_numpy(wj["v0"]).cuda()
        xo, vo = torch.empty_like(x), torch.empty_like(v)
        wo = torch.empty(150, dtype=torch.int32, device="cuda")
        so = torch.empty(150, dtype=torch.float64, device="cuda")
        ens.run_josephson(0, 300, x, v, xo, vo, wo, so)
        assert np.all(np.isfinite(ens.observables()["mean"]))
        ens.close()
