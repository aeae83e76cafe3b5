"""GPU parity of the general-coupling Kuramoto forms (Eq. 2 with a matrix K_ij).

- Coupling sums against the plain FP64 definition sum_j K_ij sin(phi_j - phi_i):
  the FP32 CUDA-core GEMM form within FP32 rounding; the BF16 tcgen05 form
  within the BF16 bound: each product carries at most two BF16 roundings
  (2^-8 relative each), so |err_i| <= 2^-7 sum_j |K_ij| + FP32 accumulation,
  with the RMS error far below that bound.
- Trajectories: the FP32 form pathwise within 1e-5 over 10^2 steps; the BF16
  form at N = 512 (the 512-oscillator slice), r(t) within 3 standard errors
  of the FP64 oracle's r(t) over the same replicas and noise.
- Full size (N = 8192, 256 replicas): sampled coupling rows against the FP64
  direct sum.
- The CTA-pair GEMM (256 x 256 tile per cluster of two CTAs, tcgen05
  cta_group::2, the default for whole tiles where the sizes allow) against
  the one-CTA GEMM: the same coupling sums and trajectories bit for bit.
- The stream-K GEMM (SDE_FLAG_GEMM_STREAM_K: the K range of all tiles split
  over every resident CTA) against the whole-tile GEMM:
  each coupling sum differs only by the FP32 rounding of the partial sums
  (at most one rounding of the running sum per K slice of 64, 2^-24 of
  sum_j |K_ij| each: below 2^-14 sum_j |K_ij| for up to 1024 slices), and both
  stay within the BF16 bound of the FP64 definition.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from gpu_util import angle_diff, ensure_built, kur_run
from paper_0903_3852_gb300 import inputs, sde

pytestmark = pytest.mark.gpu


def _ens(model, N, R, D, dt, seed, M=100):
    ensure_built()
    return sde.Ensemble.kuramoto(model, N, R, 0.0, D, dt, seed, sample_every=M)


def _direct_rows(phi, K, rows):
    """FP64 direct sums for the given receiving rows, every replica: (R, len(rows))."""
    phi = phi.astype(np.float64)
    out = np.empty((phi.shape[0], len(rows)))
    for q, i in enumerate(rows):
        out[:, q] = np.sin(phi - phi[:, i:i + 1]) @ K[i].astype(np.float64)
    return out


@pytest.mark.parametrize("model,N,R", [(sde.SDE_KURAMOTO_GENERAL_FP32, 520, 3),
                                       (sde.SDE_KURAMOTO_GENERAL, 512, 64),
                                       (sde.SDE_KURAMOTO_GENERAL, 1024, 128)])
def test_coupling_against_fp64_definition(model, N, R):
    w = inputs.kuramoto_general(n_osc=N, replicas=R, seed=2)
    ens = _ens(model, N, R, 0.02, 0.005, 1)
    ens.set_coupling(torch.from_numpy(w["Kmat"]).cuda())
    phi = torch.from_numpy(w["phi0"]).cuda()
    got = ens.coupling(phi).cpu().numpy().astype(np.float64)
    K = w["Kmat"].astype(np.float64)
    ref = np.stack([oracle.coupling_direct(w["phi0"][r].astype(np.float64), Kmat=K) for r in range(R)])
    err = np.abs(got - ref)
    absK = np.abs(K).sum(axis=1)[None, :]
    rms = math.sqrt(np.mean(err ** 2))
    print("model %d N=%d: max err %.3e, rms %.3e, bound scale %.3e" % (model, N, err.max(), rms, absK.max()))
    if model == sde.SDE_KURAMOTO_GENERAL_FP32:
        assert np.all(err <= 1e-5 * absK)
    else:
        assert np.all(err <= 2.0 ** -7 * absK + 1e-5 * absK)
        assert rms <= 2.0 ** -9 * absK.mean()


def test_fp32_general_pathwise():
    N, R, steps = 520, 2, 100
    w = inputs.kuramoto_general(n_osc=N, replicas=R, seed=3)
    ens = _ens(sde.SDE_KURAMOTO_GENERAL_FP32, N, R, 0.02, 0.005, 9, M=50)
    ens.set_coupling(torch.from_numpy(w["Kmat"]).cuda())
    phig, rg, _ = kur_run(ens, w["phi0"], w["omega"], 0, steps)
    K = w["Kmat"].astype(np.float64)
    for r in range(R):
        phio, ro = oracle.kuramoto_run(w["phi0"][r], w["omega"][r], 0.02, 0.005, 0, steps, 9, r, Kmat=K,
                                       sample_every=50)
        err = np.abs(angle_diff(phig[r], phio)) / np.maximum(1.0, np.mod(phio, 2 * np.pi))
        assert err.max() <= 1e-5
        assert np.max(np.abs(rg[:, r] - ro)) <= 2e-5


# 64 replicas: the one-CTA GEMM and separate stage kernels; 128 replicas: the
# CTA-pair GEMM with the SRK2 sub-step fused into its epilogue (the bench's
# form: staged inputs, the Philox blocks drawn ahead)
@pytest.mark.parametrize("R,flags,cluster", [(64, 0, 1), (128, sde.SDE_FLAG_FUSED, 2)])
def test_bf16_general_r_of_t_on_512_slice_within_3se(R, flags, cluster):
    N, steps, M = 512, 200, 50
    Ro = 8  # replicas the O(N^2)-per-stage oracle integrates (the GPU runs all R)
    w = inputs.kuramoto_general(n_osc=N, replicas=R, seed=4)
    ensure_built()
    ens = sde.Ensemble.kuramoto(sde.SDE_KURAMOTO_GENERAL, N, R, 0.0, 0.02, 0.005, 5, sample_every=M, flags=flags)
    assert ens.tuning()[2] == cluster
    ens.set_coupling(torch.from_numpy(w["Kmat"]).cuda())
    phig, rg_all, obs = kur_run(ens, w["phi0"], w["omega"], 0, steps)
    K = w["Kmat"].astype(np.float64)
    ro = np.stack([oracle.kuramoto_run(w["phi0"][r], w["omega"][r], 0.02, 0.005, 0, steps, 5, r, Kmat=K,
                                       sample_every=M)[1] for r in range(Ro)], axis=1)
    rg = rg_all[:, :Ro]
    R = Ro
    diff = rg - ro  # paired: same replicas, same noise
    se = np.sqrt(rg.var(axis=1, ddof=1) / R + ro.var(axis=1, ddof=1) / R)
    print("bf16 slice: max |mean dr| %.2e, max |dr| %.2e, min 3SE %.2e"
          % (np.abs(diff.mean(axis=1)).max(), np.abs(diff).max(), 3 * se[1:].min()))
    assert np.all(np.abs(rg.mean(axis=1) - ro.mean(axis=1)) <= 3 * se + 1e-12)
    assert np.abs(diff).max() <= 5e-3  # BF16 coupling: small pathwise drift of r
    assert np.allclose(obs["mean"], rg_all.mean(axis=1), atol=1e-12)


def test_bf16_and_fp32_forms_agree():
    N, R, steps = 512, 64, 100
    w = inputs.kuramoto_general(n_osc=N, replicas=R, seed=6)
    outs = []
    for model in (sde.SDE_KURAMOTO_GENERAL, sde.SDE_KURAMOTO_GENERAL_FP32):
        ens = _ens(model, N, R, 0.02, 0.005, 2, M=0)
        ens.set_coupling(torch.from_numpy(w["Kmat"]).cuda())
        outs.append(kur_run(ens, w["phi0"], w["omega"], 0, steps)[0])
    assert np.abs(angle_diff(outs[0], outs[1])).max() <= 5e-3


def test_full_size_sampled_rows():
    w = inputs.kuramoto_general()
    N, R = w["n_osc"], w["replicas"]
    ens = _ens(sde.SDE_KURAMOTO_GENERAL, N, R, w["D"], w["dt"], w["seed"])
    ens.set_coupling(torch.from_numpy(w["Kmat"]).cuda())
    got = ens.coupling(torch.from_numpy(w["phi0"]).cuda()).cpu().numpy().astype(np.float64)
    rows = list(range(0, 128, 7)) + list(range(N - 128, N, 9))  # first and last tiles
    ref = _direct_rows(w["phi0"], w["Kmat"], rows)
    err = np.abs(got[:, rows] - ref)
    absK = np.abs(w["Kmat"][rows].astype(np.float64)).sum(axis=1)[None, :]
    print("full size: max err %.3e rms %.3e" % (err.max(), math.sqrt(np.mean(err ** 2))))
    assert np.all(err <= 2.0 ** -7 * absK)
    # a short run at full size stays finite and produces r(t) rows; the bench's
    # form (the SRK2 sub-step fused into the CTA-pair GEMM, Philox blocks drawn
    # ahead) gives the same phases and r(t) bit for bit, from step 0 and from
    # a step inside a Philox block
    for n0 in (0, 6):
        phig, rg, obs = kur_run(ens, w["phi0"], w["omega"], n0, n0 + 20)
        assert np.all(np.isfinite(phig)) and obs.shape[0] == 2
        fused = sde.Ensemble.kuramoto(sde.SDE_KURAMOTO_GENERAL, N, R, 0.0, w["D"], w["dt"], w["seed"],
                                      sample_every=100, flags=sde.SDE_FLAG_FUSED)
        assert fused.tuning()[2] == 2
        fused.set_coupling(torch.from_numpy(w["Kmat"]).cuda())
        phif, rf, _ = kur_run(fused, w["phi0"], w["omega"], n0, n0 + 20)
        assert np.array_equal(phif, phig) and np.array_equal(rf, rg)
        fused.close()


def test_size_validation():
    ensure_built()
    with pytest.raises(sde.SDEError):
        sde.Ensemble.kuramoto(sde.SDE_KURAMOTO_GENERAL, 500, 64, 0.0, 0.02, 0.005, 0)
    with pytest.raises(sde.SDEError):
        sde.Ensemble.kuramoto(sde.SDE_KURAMOTO_GENERAL_FP32, 500 + 2, 3, 0.0, 0.02, 0.005, 0)
    ens = _ens(sde.SDE_KURAMOTO_GENERAL, 512, 64, 0.02, 0.005, 0)
    phi = torch.zeros((64, 512), device="cuda")
    with pytest.raises(sde.SDEError):  # no coupling matrix yet
        ens.run_kuramoto(0, 1, phi, torch.empty_like(phi), phi)


# whole pair tiles from step 0 and from step 13 (inside a Philox block: the
# fused pair GEMMs draw each next block ahead only once a whole block of the
# run lies behind it), and the stream-K GEMM
@pytest.mark.parametrize("N,R,gemm,n0", [(1024, 128, 0, 0), (1024, 128, 0, 13),
                                         (2048, 128, sde.SDE_FLAG_GEMM_STREAM_K, 0),
                                         (512, 64, 0, 0),  # one CTA per 128 x 128 tile
                                         (1024, 128, sde.SDE_FLAG_GEMM_SINGLE_CTA, 0)])
def test_fused_epilogue_equals_separate_stage_kernels(N, R, gemm, n0):
    # the SRK2 sub-step in the GEMM epilogue computes the same expression on
    # the same FP32 accumulators, with the same Gaussians, as the separate
    # stage kernels: bit-identical
    steps = 37
    w = inputs.kuramoto_general(n_osc=N, replicas=R, seed=12)
    outs = []
    for flags in (sde.SDE_FLAG_FUSED, 0):
        ensure_built()
        ens = sde.Ensemble.kuramoto(sde.SDE_KURAMOTO_GENERAL, N, R, 0.0, 0.02, 0.005, 4, sample_every=10,
                                    flags=flags | gemm)
        want = 0 if gemm == sde.SDE_FLAG_GEMM_STREAM_K else (1 if gemm or 2 * R % 256 else 2)
        assert ens.tuning()[2] == want
        ens.set_coupling(torch.from_numpy(w["Kmat"]).cuda())
        outs.append(kur_run(ens, w["phi0"], w["omega"], n0, n0 + steps))
    assert np.array_equal(outs[0][0], outs[1][0])
    assert np.array_equal(outs[0][1], outs[1][1])


@pytest.mark.parametrize("N,R", [(1024, 128), (768, 256)])
def test_cta_pair_gemm_equals_single_cta_gemm(N, R):
    # each element of D is accumulated over the same K slices in the same
    # order by both GEMMs; only the tiling over CTAs differs
    steps = 25
    w = inputs.kuramoto_general(n_osc=N, replicas=R, seed=14)
    K = torch.from_numpy(w["Kmat"]).cuda()
    phi = torch.from_numpy(w["phi0"]).cuda()
    sums, runs = [], []
    for flags in (0, sde.SDE_FLAG_GEMM_SINGLE_CTA):
        ensure_built()
        ens = sde.Ensemble.kuramoto(sde.SDE_KURAMOTO_GENERAL, N, R, 0.0, 0.02, 0.005, 4, sample_every=5,
                                    flags=flags)
        assert ens.tuning()[2] == (1 if flags else 2)
        ens.set_coupling(K)
        sums.append(ens.coupling(phi).cpu().numpy())
        runs.append(kur_run(ens, w["phi0"], w["omega"], 0, steps))
    print("pair vs single CTA: max |d sum| %.3e, max |d phi| %.3e"
          % (np.abs(sums[0] - sums[1]).max(), np.abs(runs[0][0] - runs[1][0]).max()))
    assert np.array_equal(sums[0], sums[1])
    assert np.array_equal(runs[0][0], runs[1][0]) and np.array_equal(runs[0][1], runs[1][1])


@pytest.mark.parametrize("N,R", [(2048, 128), (4096, 128)])  # tiles split in 2 and in 4
def test_stream_k_gemm_matches_whole_tiles(N, R):
    steps = 20
    w = inputs.kuramoto_general(n_osc=N, replicas=R, seed=15)
    K = torch.from_numpy(w["Kmat"]).cuda()
    phi = torch.from_numpy(w["phi0"]).cuda()
    sums, runs = {}, {}
    SK = sde.SDE_FLAG_GEMM_STREAM_K
    for flags in (SK, 0):
        ensure_built()
        ens = sde.Ensemble.kuramoto(sde.SDE_KURAMOTO_GENERAL, N, R, 0.0, 0.02, 0.005, 4, sample_every=5,
                                    flags=flags)
        if flags == SK:
            tiles = (N // 128) * (2 * R // 256)
            assert ens.tuning()[2] == 0 and ens.tuning()[1] > tiles  # stream-K over more CTAs than tiles
        else:
            assert ens.tuning()[2] == 2
        ens.set_coupling(K)
        sums[flags] = ens.coupling(phi).cpu().numpy().astype(np.float64)
        runs[flags] = kur_run(ens, w["phi0"], w["omega"], 0, steps)
    absK = np.abs(w["Kmat"].astype(np.float64)).sum(axis=1)[None, :]
    d = np.abs(sums[SK] - sums[0])
    rows = list(range(0, 128, 5)) + list(range(N - 128, N, 11))
    ref = _direct_rows(w["phi0"], w["Kmat"], rows)
    dphi = np.abs(angle_diff(runs[SK][0], runs[0][0]))
    print("stream-K vs whole tiles N=%d: max |d sum| / sum|K| %.3e, max |d phi| %.3e, max err vs FP64 %.3e"
          % (N, (d / absK).max(), dphi.max(), np.abs(sums[SK][:, rows] - ref).max()))
    assert np.all(d <= 2.0 ** -14 * absK)
    assert np.all(np.abs(sums[SK][:, rows] - ref) <= 2.0 ** -7 * absK[:, rows])
    assert dphi.max() <= 1e-5
    assert np.abs(runs[SK][1] - runs[0][1]).max() <= 1e-6
