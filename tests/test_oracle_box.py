"""Pins of the oracle's two-region box transport: the segment tally against
brute-force sampling of the segment, surface distances against ray
marching, Marsaglia's direction method against its acceptance rate and
moments, implicit capture with roulette against the closed form of the
infinite medium, weight windows against their unbiasedness, particle
balance, and the on-demand child seeds of Eq. (5)."""
import numpy as np
import pytest

from paper_2403_06362_gb300 import workloads as W

G = W.LCG_G


def lcg(oracle):
    return oracle.Lcg(m=63, pad=0, g=G, c=1)


def box(oracle, **kw):
    return W.to_oracle_box(W.box_problem(**kw), oracle)


def counts(oracle, r):
    return dict(zip(oracle.COUNT_NAMES, (int(v) for v in r["counts"])))


def test_segment_tally_matches_brute_force(oracle):
    b = box(oracle, n_histories=1, mesh=8, side=10.0, inner=(3.0, 7.0))
    rng = np.random.default_rng(0)
    h = 10.0 / 8
    for _ in range(25):
        p = rng.random(3) * 10.0
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        # keep the segment inside the box
        tmax = min(((10.0 if u[a] > 0 else 0.0) - p[a]) / u[a] for a in range(3))
        L = rng.random() * tmax
        t64, tf = oracle.box_trace(b, p, u, L, 0.75)
        assert tf.sum() == pytest.approx(0.75 * L, rel=1e-12)
        assert abs(t64.sum() * 2.0**-32 - 0.75 * L) < 1e-8
        n = 200_000
        ts = (np.arange(n) + 0.5) / n * L
        pts = p[None, :] + ts[:, None] * u[None, :]
        idx = np.clip(np.floor(pts / h).astype(int), 0, 7)
        flat = (idx[:, 2] * 8 + idx[:, 1]) * 8 + idx[:, 0]
        est = np.bincount(flat, minlength=512) * (0.75 * L / n)
        assert np.allclose(tf, est, atol=3 * 0.75 * L / n)


def test_segment_tally_along_an_axis_and_on_edges(oracle):
    b = box(oracle, n_histories=1, mesh=4, side=4.0, inner=(1.0, 3.0))
    # from the edge x = 1 along +x for 2 cm: voxels 1 and 2 get 1 cm each
    t64, tf = oracle.box_trace(b, [1.0, 0.5, 0.5], [1.0, 0.0, 0.0], 2.0, 1.0)
    assert tf[1] == 1.0 and tf[2] == 1.0 and tf.sum() == 2.0
    # from x = 3 along -x: voxels 2 and 1
    t64, tf = oracle.box_trace(b, [3.0, 0.5, 0.5], [-1.0, 0.0, 0.0], 2.0, 1.0)
    assert tf[2] == 1.0 and tf[1] == 1.0 and int(t64[1]) == 2**32


def test_surface_distance_matches_ray_marching(oracle):
    b = box(oracle, n_histories=1)
    rng = np.random.default_rng(1)
    inner = lambda q: np.all((q > 30.0) & (q < 70.0))  # noqa: E731
    for _ in range(200):
        p = rng.random(3) * 100.0
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        region = 1 if inner(p) else 0
        d, kind = oracle.box_surface_dist(b, p, u, region)
        step = 1e-3
        t = np.arange(1, int(200 / step)) * step
        q = p[None, :] + t[:, None] * u[None, :]
        out = np.any((q < 0.0) | (q > 100.0), axis=1)
        ins = np.all((q > 30.0) & (q < 70.0), axis=1)
        change = (ins != (region == 1)) | out
        first = t[np.argmax(change)]
        assert abs(d - first) <= step * 1.01
        assert kind == (2 if out[np.argmax(change)] and not (ins[np.argmax(change)] != (region == 1)) else 1)


def test_marsaglia_direction(oracle):
    L = lcg(oracle)
    rng = np.random.default_rng(2)
    us, draws = [], 0
    for x in rng.integers(0, 2**63, size=40_000, dtype=np.uint64):
        u, d = oracle.box_iso_dir(L, int(x))
        us.append(u)
        draws += d
    us = np.array(us)
    assert np.allclose(np.linalg.norm(us, axis=1), 1.0, atol=1e-15)
    n = len(us)
    assert np.all(np.abs(us.mean(0)) < 4.5 / np.sqrt(3 * n))
    assert np.all(np.abs((us**2).mean(0) - 1 / 3) < 4.5 * np.sqrt(4 / 45 / n))
    # acceptance pi/4: two draws per attempt, 8/pi draws per direction
    mean_draws = draws / n
    assert abs(mean_draws - 8 / np.pi) < 4.5 * np.sqrt(2 * 2 * (1 - np.pi / 4) / (np.pi / 4) ** 2 / n)


def test_implicit_capture_infinite_medium(oracle):
    # E[sum of w * flight] = 1 / (Sigma_t (1 - c)) in an infinite medium; an
    # unbiased roulette at tiny weights ends the histories; no splitting.
    S, c = 1.0, 0.9
    b = box(oracle, n_histories=20_000, side=1.0e5, inner=(4.0e4, 6.0e4), sigma_t=(S, S), c=(c, c),
            ww_low=(1e-6, 1e-6), ww_high=(1e30, 1e30), ww_survive=(1e-5, 1e-5), mesh=2)
    r = oracle.box_run(lcg(oracle), b)
    per = r["tally_fp"].sum() / 20_000
    cnt = counts(oracle, r)
    assert cnt["splits"] == 0 and cnt["leak_hi"] <= 100
    sd = np.sqrt(2 / (S * S * (1 - c)) * 1 / (1 - c)) / np.sqrt(20_000)
    assert abs(per - 1.0 / (S * (1 - c))) < 4.5 * sd + 0.002 * per


def test_weight_windows_are_unbiased(oracle):
    # the same problem with and without windows estimates the same flux
    base = dict(n_histories=40_000, mesh=4)
    r1 = oracle.box_run(lcg(oracle), box(oracle, **base))
    r0 = oracle.box_run(lcg(oracle), box(oracle, ww_low=(1e-6, 1e-6), ww_high=(1e30, 1e30),
                                         ww_survive=(1e-5, 1e-5), **base))
    c1 = counts(oracle, r1)
    assert c1["splits"] > 0 and c1["roulette_kills"] > 0
    t1, t0 = r1["tally_fp"].sum() / 40_000, r0["tally_fp"].sum() / 40_000
    # per-history weighted track length has sd < 40 cm here
    assert abs(t1 - t0) < 4.5 * 40 * np.sqrt(2 / 40_000)


def test_particle_balance_and_children(oracle):
    r = oracle.box_run(lcg(oracle), box(oracle, n_histories=5000))
    c = counts(oracle, r)
    assert c["source"] + c["children"] == c["leak_hi"] + c["roulette_kills"] + c["capped"]
    assert c["children"] >= c["splits"] > 0
    assert c["collisions"] == c["scatters"] and c["absorptions"] == 0


def test_child_seed_is_eq5(oracle):
    # A split's children are seeded with hash(k, S_p): run histories one by
    # one; the family of history i depends on nothing but its own seed, so
    # any split of the id range adds up to the same int64 tally.
    b = box(oracle, n_histories=3000)
    L = lcg(oracle)
    whole = oracle.box_run(L, b)
    t = np.zeros_like(whole["tally"])
    cnt = np.zeros_like(whole["counts"])
    for a, e in [(0, 1000), (1000, 1001), (1001, 3000)]:
        oracle.box_run(L, b, a, e, tally=t, counts=cnt)
    assert np.array_equal(t, whole["tally"])
    assert np.array_equal(cnt[:13], whole["counts"][:13])


def test_box_seeds(oracle):
    L = lcg(oracle)
    b = box(oracle, n_histories=10)
    assert oracle.box_seed(L, b, 5) == oracle.hash_seed(5, 42, 63)
    bs = box(oracle, n_histories=10, seeding=W.SEED_STRIDE)
    assert oracle.box_seed(L, bs, 5) == oracle.stride_seed(1, W.STRIDE_Q, 5, 63, G, 1)


def test_group_choice_follows_the_cdf_rows(oracle):
    """Downscatter (R18): the group picked for u uniform on [0, 1) is g' with
    probability CDF[g'] - CDF[g' - 1] (chi-square per row), and a u on a row
    boundary belongs to the next group (u < CDF strictly)."""
    from scipy.stats import chi2
    P = W.to_oracle_box(W.box_problem(n_histories=1), oracle)
    us = np.random.default_rng(11).random(40000)
    for rg in range(2):
        for g in range(int(P.n_groups)):
            cdf = np.array([P.cdf[rg][g][k] for k in range(int(P.n_groups))])
            prob = np.diff(np.concatenate([[0.0], cdf]))
            picks = np.array([oracle.box_next_group(P, rg, g, float(u)) for u in us])
            assert picks.min() >= g  # downscatter only
            obs = np.bincount(picks, minlength=len(prob)).astype(float)
            live = prob > 0
            stat = np.sum((obs[live] - len(us) * prob[live]) ** 2 / (len(us) * prob[live]))
            assert chi2.sf(stat, max(int(live.sum()) - 1, 1)) > 1e-4, (rg, g, obs, prob)
            for k in range(g, int(P.n_groups) - 1):
                if cdf[k] > 0:
                    assert oracle.box_next_group(P, rg, g, float(cdf[k])) > k


def test_mesh_tally_is_symmetric(oracle):
    """The box, its inner cube, the uniform isotropic source and the weight
    windows are symmetric under axis permutations and under x -> side - x,
    so the expected mesh tally is too: the three axis profiles agree, and
    each equals its mirror image, within batch errors."""
    b = W.box_problem(n_histories=6000, seeding=W.SEED_HASH, n_batches=12)
    L = oracle.Lcg(m=63, pad=0, g=W.LCG_G, c=1)
    t = oracle.box_run(L, W.to_oracle_box(b, oracle))["tally"].astype(np.float64)
    nm = b["mesh"]
    t = t.reshape(12, nm, nm, nm)  # [batch][z][y][x]
    prof = {"x": t.sum(axis=(1, 2)), "y": t.sum(axis=(1, 3)), "z": t.sum(axis=(2, 3))}  # [batch][i]

    def close(a, c):
        d = a - c  # per batch, per bin
        se = d.std(axis=0, ddof=1) / np.sqrt(d.shape[0])
        z = d.mean(axis=0) / np.where(se > 0, se, np.inf)
        return np.abs(z).max()

    assert close(prof["x"], prof["y"]) < 5.0
    assert close(prof["x"], prof["z"]) < 5.0
    for ax in "xyz":
        assert close(prof[ax], prof[ax][:, ::-1]) < 5.0
