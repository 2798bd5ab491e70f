"""Shared helpers of the GPU parity tests (host side, oracle only)."""
import numpy as np


def accounted_pair(oracle_lib, s, params, src, tgt, Xi, Xj, gpu_mask, r):
    """oracle.accounted_pair: the oracle's pair sums with the GPU's other-way
    decisions moved to the GPU's side; (H, b, cost, count, n_flipped,
    n_unexplained)."""
    return oracle_lib.accounted_pair(s, params, src, tgt, Xi, Xj, gpu_mask, r)


def _pair_job(args):
    """One sampled pair on an oracle worker: the oracle's pair sums, its mask and
    flags, and the sums with the GPU's other-way decisions accounted for."""
    import oracle
    s, params, src, tgt, Xi, Xj, gpu_mask = args
    r = oracle.linearize_pair(s, params, src, tgt, Xi, Xj)
    n = r["n_points"]
    m = gpu_mask[: len(r["mask"])]
    acc = accounted_pair(oracle, s, params, src, tgt, Xi, Xj, m, r)
    return dict(n_points=n, count=r["count"], mask=r["mask"], flags=r["flags"], acc=acc)


# Bars of the sampled large configurations.  The sub-system of the sampled
# pairs (their blocks side by side) meets the bars of the iteration's system
# (H, b 1e-4, cost 1e-5); each pair alone meets SUB_PAIR_BAR on H and b and
# 1e-4 on its cost.  A float32 pixel-point at 40-80 m is stored to ~4e-6 m,
# i.e. its projection to ~3e-5 px, and at a depth discontinuity the sampled
# depth changes by tens of metres per pixel, so e_d (and through it the Huber
# weight) of such points moves by up to ~1e-3 relative; a pair whose system is
# dominated by a few of them reaches ~1e-4 alone, while the sum over pairs
# stays well inside 1e-4.
SUB_PAIR_BAR = 1e-3


def check_sampled_pairs(oracle_lib, w, p, n_sample, seed, params, host, rel, workers=None):
    """Linearise on the GPU with mask export, then recompute a seeded sample of
    n_sample pairs with the oracle (in spawn-started worker processes: safe
    after CUDA initialisation) and check, against the oracle's sums with the
    points decided the other way accounted for: per pair, the masks outside
    the oracle's decision margin, the count, H12 / b12 to SUB_PAIR_BAR and the
    cost to 1e-4; over the sample, the stacked blocks' H and b to 1e-4 and the
    summed cost to 1e-5 (relative Frobenius), and at most 1e-5 of the
    residuals (+2) decided the other way at all.  Returns (pairs checked,
    residuals, points decided the other way)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    import os
    p.set_mask_export(True)
    p.linearize()
    ps = p.get_pair_system()
    rng = np.random.default_rng(seed)
    sample = rng.choice(len(w.pairs), size=min(n_sample, len(w.pairs)), replace=False).tolist()
    jobs = []
    for q in sample:
        i, j = w.pairs[q].tolist()
        s = w.sensors[int(w.frame_sensor[i])]
        n_pts = p.frame_points(i)
        jobs.append((s, params, host(w.channels[i]), host(w.channels[j]), w.poses_init[i], w.poses_init[j],
                     p.get_mask(q, n_pts)))
    n_workers = workers or max(1, min(len(jobs), (os.cpu_count() or 2) - 1))
    with cf.ProcessPoolExecutor(n_workers, mp_context=mp.get_context("spawn")) as ex:
        results = list(ex.map(_pair_job, jobs))
    residuals, flipped = 0, 0
    dH2 = H2 = db2 = b2 = dc = c = 0.0
    for q, job, r in zip(sample, jobs, results):
        m = job[-1]
        assert p.frame_points(w.pairs[q][0]) == r["n_points"], q
        assert not np.any((m ^ r["mask"]) & ~r["flags"]), f"pair {q}: masks differ outside the decision margin"
        Ho, bo, co, no, nf, nu = r["acc"]
        assert nu == 0, f"pair {q}: {nu} flipped points without an other-branch evaluation"
        assert int(ps["count"][q]) == no, q
        assert rel(ps["H"][q], Ho) <= SUB_PAIR_BAR, (q, nf, rel(ps["H"][q], Ho))
        assert rel(ps["b"][q], bo) <= SUB_PAIR_BAR, (q, nf, rel(ps["b"][q], bo))
        assert abs(ps["cost"][q] - co) <= 1e-4 * co + 1e-12, q
        dH2 += float(np.sum((ps["H"][q] - Ho) ** 2))
        H2 += float(np.sum(Ho ** 2))
        db2 += float(np.sum((ps["b"][q] - bo) ** 2))
        b2 += float(np.sum(bo ** 2))
        dc += abs(float(ps["cost"][q]) - co)
        c += co
        residuals += r["count"]
        flipped += nf
    assert (dH2 / H2) ** 0.5 <= 1e-4 and (db2 / b2) ** 0.5 <= 1e-4, ((dH2 / H2) ** 0.5, (db2 / b2) ** 0.5)
    assert dc <= 1e-5 * c, dc / c
    assert flipped <= 1e-5 * residuals + 2, (flipped, residuals)
    p.set_mask_export(False)
    return len(sample), residuals, flipped
