"""Shared helpers of the GPU parity tests (host side, oracle only)."""
import numpy as np


def accounted_pair(oracle_lib, s, params, src, tgt, Xi, Xj, gpu_mask, r):
    """The oracle's sums of one pair with every flagged point that the GPU
    decided the other way moved to the GPU's side: its contribution (from the
    oracle, or from the oracle's other-branch evaluation when the oracle
    rejected it) is removed or added.  Returns (H, b, cost, count, n_flipped,
    n_unexplained)."""
    H, b, cost, count = r["H"].copy(), r["b"].copy(), r["cost"], r["count"]
    n = r["n_points"]
    diff = np.unpackbits((gpu_mask ^ r["mask"]).view(np.uint8), bitorder="little")[:n]
    ok_o = np.unpackbits(r["mask"].view(np.uint8), bitorder="little")[:n]
    idx = np.nonzero(diff)[0]
    unexplained = 0
    if idx.size:
        pts, _ = oracle_lib.frame_points(s, params, src)
        for k in idx.tolist():
            c = oracle_lib.point_contribution(s, params, tgt, Xi, Xj, pts[k], other_branch=not ok_o[k])
            if c is None:
                unexplained += 1
                continue
            sign = -1.0 if ok_o[k] else 1.0
            H += sign * c[0]
            b += sign * c[1]
            cost += sign * c[2]
            count += int(sign)
    return H, b, cost, count, int(idx.size), unexplained


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


def check_sampled_pairs(oracle_lib, w, p, n_sample, seed, params, host, rel, workers=None):
    """Linearise on the GPU with mask export, then recompute a seeded sample of
    n_sample pairs with the oracle (in spawn-started worker processes: safe
    after CUDA initialisation) and check, per pair, the masks outside the
    oracle's decision margin, H12 / b12 to 1e-4 and the cost to 1e-5 against
    the oracle's sums with the points decided the other way accounted for;
    over the sample, at most 1e-5 of the residuals (+2) may be decided the
    other way at all.  Returns (pairs checked, residuals, points decided the
    other way)."""
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
    for q, job, r in zip(sample, jobs, results):
        m = job[-1]
        assert p.frame_points(w.pairs[q][0]) == r["n_points"], q
        assert not np.any((m ^ r["mask"]) & ~r["flags"]), f"pair {q}: masks differ outside the decision margin"
        Ho, bo, co, no, nf, nu = r["acc"]
        assert nu == 0, f"pair {q}: {nu} flipped points without an other-branch evaluation"
        assert int(ps["count"][q]) == no, q
        assert rel(ps["H"][q], Ho) <= 1e-4, (q, nf, rel(ps["H"][q], Ho))
        assert rel(ps["b"][q], bo) <= 1e-4, (q, nf, rel(ps["b"][q], bo))
        assert abs(ps["cost"][q] - co) <= 1e-5 * co + 1e-12, q
        residuals += r["count"]
        flipped += nf
    assert flipped <= 1e-5 * residuals + 2, (flipped, residuals)
    p.set_mask_export(False)
    return len(sample), residuals, flipped
