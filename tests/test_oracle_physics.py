"""Physics pins of the oracle: samplers against analytic distributions, transport against
closed forms, single interactions against kinematic identities, runs against invariants."""
import numpy as np
import pytest
from scipy import integrate, stats

import oracle
from paper_2302_08252_gb300 import workloads as W

MC2 = 0.51099895
KC = 0.01


def kn_dsig_deps(eps, k):
    """Textbook Klein-Nishina dsigma/deps (up to the constant pi r_e^2 / k)."""
    cost = 1.0 - (1.0 - eps) / (k * eps)
    return eps + 1.0 / eps - (1.0 - cost * cost)


@pytest.mark.parametrize("k", [0.02, 0.2, 2.0, 20.0, 2000.0])
def test_klein_nishina_sampler_chi2(k):
    n = 200_000
    ids = np.arange(n, dtype=np.uint64) + (np.uint64(9) << np.uint64(32))
    eps, att = oracle.compton_eps(k, ids, seed=11, event=3, step=5)
    assert att.max() < 64
    e0 = 1.0 / (1.0 + 2.0 * k)
    edges = np.linspace(e0, 1.0, 51)
    obs, _ = np.histogram(eps.astype(np.float64), bins=edges)
    w = np.array([integrate.quad(kn_dsig_deps, a, b, args=(k,), epsrel=1e-11)[0]
                  for a, b in zip(edges[:-1], edges[1:])])
    exp = n * w / w.sum()
    chi2 = ((obs - exp) ** 2 / exp).sum()
    p = stats.chi2.sf(chi2, df=49)
    assert p > 1e-3, (chi2, p)


def _photon(world, e, d=(0.0, 0.0, 1.0), nia=0.0, id=0, slab=0, z=None, x=0.0, y=0.0):
    z = world_plane(world, slab) + 0.5 if z is None else z
    return oracle.make_track(x=x, y=y, z=z, d=d, e=e, nia=nia, id=id, slab=slab)


def world_plane(world, slab):
    return float(np.cumsum(np.concatenate([[0.0], world._keep[0]]))[slab])


def _unit(rng, n):
    v = rng.normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def test_brem_spectrum_ks(oworld):
    t0 = 1000.0
    ks = []
    for i in range(20000):
        r = oracle.step_one(oworld, W.E_MINUS, _photon(oworld, t0, id=i))
        assert r["proc"] == oracle.PROC_BREM and r["lim"] == oracle.LIM_PHYS
        assert r["sec_type"][0] == W.GAMMA
        k = float(r["sec"][0]["e"])
        assert KC <= k <= t0
        assert r["track"]["e"] == np.float32(np.float32(t0) - np.float32(k))
        ks.append(k)
    ks = np.array(ks)
    cdf = lambda k: np.log(k / KC) / np.log(t0 / KC)
    assert stats.kstest(ks, cdf).pvalue > 1e-3


def test_compton_kinematics_and_azimuth(oworld):
    rng = np.random.default_rng(5)
    dirs = _unit(rng, 6000)
    phis, n_c = [], 0
    for i, d in enumerate(dirs):
        e = 2.0
        r = oracle.step_one(oworld, W.GAMMA, _photon(oworld, e, d=tuple(d), id=i))
        if r["proc"] != oracle.PROC_COMPTON:
            continue
        n_c += 1
        t = r["track"]
        e1 = float(t["e"])
        d1 = np.array([t["dx"], t["dy"], t["dz"]], np.float64)
        d0 = np.array(d, np.float32).astype(np.float64)
        cos_k = 1.0 - MC2 * (1.0 / e1 - 1.0 / e)       # Compton formula
        assert np.dot(d0, d1) == pytest.approx(cos_k, abs=2e-5)
        assert np.linalg.norm(d1) == pytest.approx(1.0, abs=2e-6)
        if r["nsec"]:
            s = r["sec"][0]
            de = np.array([s["dx"], s["dy"], s["dz"]], np.float64)
            assert float(s["e"]) == pytest.approx(e - e1, rel=1e-6)
            p = e * d0 - e1 * d1
            assert np.dot(de, p / np.linalg.norm(p)) == pytest.approx(1.0, abs=1e-5)
        # azimuth of d1 about d0 in a fixed frame
        a = np.cross(d0, [0.0, 0.0, 1.0] if abs(d0[2]) < 0.9 else [1.0, 0.0, 0.0])
        a /= np.linalg.norm(a)
        b = np.cross(d0, a)
        perp = d1 - np.dot(d1, d0) * d0
        if np.linalg.norm(perp) > 1e-3:
            phis.append(np.arctan2(np.dot(perp, b), np.dot(perp, a)))
    assert n_c > 3000
    phis = (np.array(phis) + np.pi) / (2 * np.pi)
    assert stats.kstest(phis, "uniform").pvalue > 1e-3


def test_photon_process_fractions(oworld):
    # at 20 MeV in lead all three processes compete; fractions follow the cross sections
    e, n = 20.0, 20000
    procs = np.array([oracle.step_one(oworld, W.GAMMA, _photon(oworld, e, id=i))["proc"]
                      for i in range(n)])
    sc, sp, se = (oracle.sigma(k, 0, e) for k in ("compton", "pair", "phot"))
    tot = sc + sp + se
    for proc, s in ((oracle.PROC_COMPTON, sc), (oracle.PROC_PAIR, sp), (oracle.PROC_PHOT, se)):
        f = np.mean(procs == proc)
        p = s / tot
        assert abs(f - p) < 4 * np.sqrt(p * (1 - p) / n) + 2e-3 * p, (proc, f, p)


def test_pair_and_photoelectric_kinematics(oworld):
    for i in range(3000):
        e = 50.0
        r = oracle.step_one(oworld, W.GAMMA, _photon(oworld, e, id=i))
        if r["proc"] == oracle.PROC_PAIR:
            assert r["alive"] == 0 and r["death"] == oracle.DEATH_ABSORB
            es = sum(float(s["e"]) for s in r["sec"] if s["e"] != np.float32(MC2)) + r["cut"]
            assert es == pytest.approx(e - 2 * MC2, rel=1e-6)
            assert r["mc"] == pytest.approx(2 * MC2, rel=1e-5)
            for s, ty in zip(r["sec"], r["sec_type"]):
                if ty != W.GAMMA:
                    assert (s["dx"], s["dy"], s["dz"]) == (0.0, 0.0, 1.0)
        elif r["proc"] == oracle.PROC_PHOT:
            assert r["nsec"] == 1 and r["sec_type"] == [W.E_MINUS]
            assert r["sec"][0]["e"] == np.float32(e)
    # low energy in lead: photoelectric dominates
    r = oracle.step_one(oworld, W.GAMMA, _photon(oworld, 0.02, id=1))
    assert r["proc"] == oracle.PROC_PHOT


def test_annihilation_at_rest(oworld):
    # a 0.5 MeV positron ranges out in one step (loss limit), then annihilates at rest
    for i in range(200):
        tr = _photon(oworld, 0.5, nia=50.0, id=i)
        r = oracle.step_one(oworld, W.E_PLUS, tr)
        assert r["lim"] == oracle.LIM_LOSS and r["death"] == oracle.DEATH_CUT
        assert r["nsec"] == 2 and r["sec_type"] == [W.GAMMA, W.GAMMA]
        a, b = r["sec"]
        assert a["e"] == b["e"] == np.float32(MC2)
        da = np.array([a["dx"], a["dy"], a["dz"]])
        db = np.array([b["dx"], b["dy"], b["dz"]])
        assert np.array_equal(da, -db)
        assert np.linalg.norm(da) == pytest.approx(1.0, abs=1e-6)
        assert r["mcr"] == 2 * float(np.float32(MC2))
        assert r["dep_cont"] == float(np.float32(0.5))    # the whole kinetic energy


def _block_uniforms(track_id: int, step: int, block: int, seed: int = 1, event: int = 0):
    """The four uniforms of Philox block `block` of a track's step, from the KAT-pinned
    Philox and the endpoint-pinned u01 conversion (the keying of the toy model's draws)."""
    ctr = np.array([[track_id & 0xFFFFFFFF, track_id >> 32, step, block]], dtype=np.uint32)
    return [oracle.u01(int(x)) for x in oracle.philox(ctr, (seed, event))[0]]


def test_pair_energy_share_uniform(oworld):
    # a 1 GeV photon in lead almost always pair-produces; the electron's share of the
    # kinetic energy left after the two rest masses is uniform on [0, 1] and comes from
    # the third uniform of the step's draw block
    e = np.float32(1000.0)
    avail = np.float32(e - np.float32(2 * MC2))
    share, n_pair = [], 0
    for i in range(12000):
        r = oracle.step_one(oworld, W.GAMMA, _photon(oworld, float(e), id=i))
        if r["proc"] != oracle.PROC_PAIR:
            continue
        n_pair += 1
        em = [s["e"] for s, ty in zip(r["sec"], r["sec_type"]) if ty == W.E_MINUS]
        if not em:  # electron below the cut: its energy went to the below-cut tally
            continue
        u = _block_uniforms(i, 0, 0)
        assert em[0] == np.float32(np.float32(u[2]) * avail), i
        share.append(float(em[0]) / float(avail))
    assert n_pair >= 10000
    assert stats.kstest(share, "uniform").pvalue > 1e-3
    # the share does not depend on the process-selection draw (a reused u1 would
    # confine it to the pair's sub-interval of [0, 1])
    lo = np.asarray(share) < 0.5
    assert 0.45 < lo.mean() < 0.55


def test_annihilation_angles_isotropic(oworld):
    # the photon pair of a positron annihilating at rest is isotropic: cos(theta) uniform on
    # [-1, 1], phi uniform on [0, 2 pi), the two independent; drawn from block 65 of the
    # positron's last step (first uniform -> cos(theta), second -> phi)
    n = 10000
    cost = np.empty(n)
    phi = np.empty(n)
    for i in range(n):
        r = oracle.step_one(oworld, W.E_PLUS, _photon(oworld, 0.5, nia=50.0, id=i))
        assert r["nsec"] == 2
        a = r["sec"][0]
        cost[i] = float(a["dz"])
        phi[i] = np.arctan2(float(a["dy"]), float(a["dx"])) % (2 * np.pi)
        u = _block_uniforms(i, 0, 65)
        assert a["dz"] == np.float32(np.float32(2.0) * np.float32(u[0]) - np.float32(1.0)), i
        d = abs(phi[i] - 2 * np.pi * u[1])
        if abs(float(a["dz"])) < 0.999:  # phi is ill-defined at the poles
            assert min(d, 2 * np.pi - d) < 1e-4, (i, phi[i], u[1])
    assert stats.kstest(cost, "uniform", args=(-1.0, 2.0)).pvalue > 1e-3
    assert stats.kstest(phi, "uniform", args=(0.0, 2 * np.pi)).pvalue > 1e-3
    # independence: chi-square of the 5 x 5 contingency table of (cos theta, phi)
    h, _, _ = np.histogram2d(cost, phi, bins=[np.linspace(-1, 1, 6),
                                             np.linspace(0, 2 * np.pi, 6)])
    assert stats.chi2_contingency(h)[1] > 1e-3


# ---- toy model v2: multiple scattering of e+- ----

MSC_FR, MSC_RMIN = 0.04, 0.5     # step limit: F_R max(E / dEdx, R_MIN), mm
X0_PB, X0_LAR = 5.612, 140.0     # mm


def highland_theta0(e_mev, s_mm, x0_mm):
    """Highland's width of the projected scattering angle (PDG, Lynch and Dahl form):
    13.6 MeV / (beta c p) sqrt(x) (1 + 0.038 ln x), x = s / X0, z = 1."""
    pbc = e_mev * (e_mev + 2 * MC2) / (e_mev + MC2)  # (pc)^2 / E_total
    x = s_mm / x0_mm
    return 13.6 / pbc * np.sqrt(x) * (1.0 + 0.038 * np.log(x))


@pytest.fixture(scope="module")
def msc_world(otables):
    return oracle.World(W.single_slab(5000.0, material=0), otables, seed=1, msc=True)


@pytest.mark.parametrize("e", [0.1, 0.3, 1.0, 5.0, 50.0, 500.0])
def test_msc_step_limit(msc_world, e):
    # in a thick lead slab, with no interaction due, a charged step is limited by
    # multiple scattering to F_R max(E / dEdx, R_MIN) (always below the loss limit)
    for ptype in (W.E_MINUS, W.E_PLUS):
        r = oracle.step_one(msc_world, ptype, oracle.make_track(z=0.0, e=e, nia=1e6, slab=0))
        assert r["lim"] == oracle.LIM_MSC
        rng = e / 1.274
        assert float(r["track"]["len"]) == pytest.approx(MSC_FR * max(rng, MSC_RMIN), rel=1e-6)
    # photons are not scattered
    r = oracle.step_one(msc_world, W.GAMMA, oracle.make_track(z=0.0, e=e, nia=1e6, slab=0))
    assert r["lim"] == oracle.LIM_Z and (r["track"]["dx"], r["track"]["dy"]) == (0.0, 0.0)


def test_msc_v1_unchanged(oworld, otables):
    # the v1 world takes the same steps as before: no scattering limit, no deflection
    w1 = oracle.World(W.single_slab(5000.0, material=0), otables, seed=1, msc=False)
    r = oracle.step_one(w1, W.E_MINUS, oracle.make_track(z=0.0, e=50.0, nia=1e6, slab=0))
    assert r["lim"] == oracle.LIM_LOSS
    assert (r["track"]["dx"], r["track"]["dy"], r["track"]["dz"]) == (0.0, 0.0, 1.0)


@pytest.mark.parametrize("e,mat", [(20.0, 0), (100.0, 0), (1000.0, 0), (100.0, 1)])
def test_msc_deflection_highland(otables, e, mat):
    # after one scattering-limited step along +z, 1 - cos(theta) over theta0^2 (Highland
    # at the step's own length, FP64) is exponential with mean 1 (the small-angle Gaussian
    # law: theta^2 / 2 has mean theta0^2), the azimuth is uniform, and both come from
    # Philox block 66 of the step (first uniform -> theta, second -> phi)
    msc_world = oracle.World(W.single_slab(5000.0, material=mat), otables, seed=1, msc=True)
    x0, dedx = (X0_PB, 1.274) if mat == 0 else (X0_LAR, 0.2105)
    n = 20000
    w = np.empty(n)
    phi = np.empty(n)
    s = None
    for i in range(n):
        r = oracle.step_one(msc_world, W.E_MINUS,
                            oracle.make_track(z=0.0, e=e, nia=1e6, slab=0, id=i))
        t = r["track"]
        assert r["lim"] == oracle.LIM_MSC and r["alive"]
        s = float(t["len"]) if s is None else s
        d = np.array([t["dx"], t["dy"], t["dz"]], dtype=np.float64)
        assert np.linalg.norm(d) == pytest.approx(1.0, abs=2e-6)
        w[i] = 1.0 - d[2]
        phi[i] = np.arctan2(d[1], d[0]) % (2 * np.pi)
        if i < 500:
            u = _block_uniforms(i, 0, 66)
            th0 = highland_theta0(e, s, x0)
            assert w[i] == pytest.approx(th0 * th0 * -np.log(u[0]), rel=2e-3, abs=1e-6), i
            dphi = abs(phi[i] - 2 * np.pi * u[1])
            assert min(dphi, 2 * np.pi - dphi) < 1e-3, i
    th0 = highland_theta0(e, s, x0)
    assert stats.kstest(w / th0**2, "expon").pvalue > 1e-3
    assert np.mean(w) / th0**2 == pytest.approx(1.0, abs=4.0 / np.sqrt(n))
    assert stats.kstest(phi, "uniform", args=(0.0, 2 * np.pi)).pvalue > 1e-3
    # the step length the width was computed for
    assert s == pytest.approx(MSC_FR * e / dedx, rel=1e-6)


def test_msc_width_scales_with_thickness(otables):
    # a 1 GeV electron crossing a lead slab of exactly one radiation length into the next
    # (the geometry limit wins: F_R E / dEdx = 31 mm): ln x = 0, so theta0 is
    # 13.6 MeV / (beta c p) exactly
    slab = {"thickness": np.array([X0_PB, 100.0]), "material": np.array([0, 0], np.uint8),
            "half_xy": 1.0e6}
    wld = oracle.World(slab, otables, seed=1, msc=True)
    n = 20000
    w = np.empty(n)
    for i in range(n):
        r = oracle.step_one(wld, W.E_MINUS,
                            oracle.make_track(z=0.0, e=1000.0, nia=1e6, slab=0, id=i))
        assert r["lim"] == oracle.LIM_Z
        w[i] = 1.0 - float(r["track"]["dz"])
    pbc = 1000.0 * (1000.0 + 2 * MC2) / (1000.0 + MC2)
    th0 = 13.6 / pbc
    assert stats.kstest(w / th0**2, "expon").pvalue > 1e-3


def test_msc_run_invariants(geom, otables):
    p = W.small_electrons()
    r1 = oracle.run(geom, p, seed=1, tables=otables)
    r2 = oracle.run(geom, p, seed=1, tables=otables, msc=True, idlog=True)
    assert _ledger_rel(r2) < 1e-12
    c = r2["counts"].astype(np.int64)
    assert np.array_equal(c.sum(0), r2["steps"].astype(np.int64))
    assert len(r2["idlog"]) == int(r2["tracks"].sum())
    # more charged steps, the same photon physics; the showers stay contained
    assert r2["steps"][0] > 3 * r1["steps"][0] and r2["steps"][1] > 3 * r1["steps"][1]
    assert r2["score"].sum() > 0.95 * 16 * 1000.0


def test_msc_fp64_reference_agrees_with_strict(geom, otables):
    p = W.mixed_primaries(400)
    p["ekin"] = np.minimum(p["ekin"], np.float32(2000.0))
    n = 400
    r32 = oracle.run(geom, p, n_events=n, seed=1, tables=otables, msc=True, nthreads=8)
    r64 = oracle.run(geom, p, n_events=n, seed=1, tables=otables, msc=True, nthreads=8,
                     mode=oracle.REF_FP64)
    a = r32["score"].reshape(n, -1, 2).sum(2)
    b = r64["score"].reshape(n, -1, 2).sum(2)
    se = np.sqrt(a.var(0, ddof=1) / n + b.var(0, ddof=1) / n)
    d = np.abs(a.mean(0) - b.mean(0))
    assert np.all(d <= 3 * se + 1e-9)
    big = b.mean(0) >= 0.01 * b.mean(0).sum()
    assert np.all(d[big] / b.mean(0)[big] <= 0.01)


def test_geometry_limits(oworld):
    # photon along +z from the front face: stops exactly on the first plane, enters slab 1
    tr = oracle.make_track(z=0.0, d=(0.0, 0.0, 1.0), e=1.0, nia=1e6, slab=0)
    r = oracle.step_one(oworld, W.GAMMA, tr)
    t = r["track"]
    assert r["lim"] == oracle.LIM_Z and t["z"] == np.float32(2.3) and t["slab"] == 1
    assert t["len"] == np.float32(2.3)
    assert t["time"] == np.float32(np.float32(2.3) / np.float32(299.792458))
    # backwards out of slab 0: escapes with its energy
    tr = oracle.make_track(z=1.0, d=(0.0, 0.0, -1.0), e=3.0, nia=1e6, slab=0)
    r = oracle.step_one(oworld, W.GAMMA, tr)
    assert r["death"] == oracle.DEATH_ESCAPE and r["esc"] == 3.0
    # sideways through the +x face
    tr = oracle.make_track(x=199.0, z=1.0, d=(1.0, 0.0, 0.0), e=3.0, nia=1e6, slab=0)
    r = oracle.step_one(oworld, W.GAMMA, tr)
    assert r["lim"] == oracle.LIM_X and r["death"] == oracle.DEATH_ESCAPE
    assert r["track"]["x"] == np.float32(200.0)
    # a 100 MeV electron in lead takes the 20% energy-loss step
    tr = oracle.make_track(z=0.1, d=(0.6, 0.0, 0.8), e=100.0, nia=1e6, slab=0)
    r = oracle.step_one(oworld, W.E_MINUS, tr)
    s = np.float32(np.float32(0.2) * np.float32(100.0)) / np.float32(1.274)
    # the z plane at 2.3 mm is reached after 2.75 mm, the loss limit at 15.7 mm
    assert r["lim"] == oracle.LIM_Z
    tr = oracle.make_track(z=0.1, d=(0.0, 0.0, 1.0), e=100.0, nia=1e6, slab=0)
    wide = oracle.World(W.single_slab(1000.0), oworld.tables, seed=1)
    r = oracle.step_one(wide, W.E_MINUS, tr)
    assert r["lim"] == oracle.LIM_LOSS and r["track"]["len"] == s


def test_range_closed_form(otables):
    # brems switched off: an electron loses T0 continuously over the range T0/dEdx
    t = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in otables.items()}
    t["sig32"][:, oracle.TAB_BREM] = 0
    t["sig64"][:, oracle.TAB_BREM] = 0
    w = oracle.World(W.single_slab(5000.0, material=0), t, seed=1)
    t0 = 50.0
    tr = oracle.make_track(z=0.0, e=t0, slab=0)
    dep, n = 0.0, 0
    while True:
        r = oracle.step_one(w, W.E_MINUS, tr)
        dep += r["dep_cont"] + r["cut"]
        n += 1
        if not r["alive"]:
            break
        tr = np.array([r["track"]], dtype=oracle.TRACK32_DTYPE)
    assert dep == pytest.approx(t0, rel=1e-12)
    assert float(r["track"]["len"]) == pytest.approx(t0 / float(np.float32(1.274)), rel=1e-5)
    assert n == 19    # 18 steps of 20% loss (50 * 0.8^18 < 1 MeV) and the range-out step


def test_attenuation_unscattered_fraction(otables):
    e, L, n = 1.0, 10.0, 20000
    geom = W.single_slab(L, material=0)
    p = W.gun(n, e, ptype=W.GAMMA)
    r = oracle.run(geom, p, seed=4, idlog=True, tables=otables)
    log = r["idlog"]
    prim = (log["id"] & np.uint64(0xFFFFFFFF)) == 0
    death = log["type_death"] >> 8
    through = prim & (log["steps"] == 1) & (death == oracle.DEATH_ESCAPE)
    frac = through.sum() / n
    sig = sum(oracle.sigma(k, 0, e) for k in ("compton", "pair", "phot"))
    pexp = np.exp(-sig * L)
    assert abs(frac - pexp) < 4 * np.sqrt(pexp * (1 - pexp) / n) + 1e-3


def _ledger_rel(r):
    L = r["ledger"]
    src = L[:, 0] + L[:, 4]
    snk = L[:, 1] + L[:, 2] + L[:, 3] + L[:, 5]
    return np.max(np.abs(src - snk) / src)


def test_run_invariants_small_electrons(geom, otables):
    p = W.small_electrons()
    r = oracle.run(geom, p, seed=1, idlog=True, tables=otables)
    assert _ledger_rel(r) < 1e-12
    L = r["ledger"]
    assert np.allclose(r["score"].sum(1), L[:, 1] + L[:, 2], rtol=1e-12, atol=0)
    assert np.all(L[:, 0] == 1000.0)
    c = r["counts"].astype(np.int64)
    assert list(c[0]) == [16, 0, 0]
    assert c.sum() == int(r["steps"].sum())
    assert np.array_equal(c.sum(0), r["steps"].astype(np.int64))
    log = r["idlog"]
    assert len(log) == int(r["tracks"].sum())
    assert len(np.unique(log["id"])) == len(log)
    assert int(log["steps"].astype(np.int64).sum()) == int(r["steps"].sum())
    assert np.array_equal(np.bincount(log["type_death"] & 0xFF, minlength=3),
                          r["tracks"].astype(np.int64))
    # a 1 GeV shower in 22 X0 deposits nearly all its energy
    assert 0.95 < (r["score"].sum(1) / L[:, 0]).mean() <= 1.0


def test_run_invariants_mixed_types(geom, otables):
    p = W.mixed_primaries(60)
    p["ekin"] = np.minimum(p["ekin"], np.float32(3000.0))
    r = oracle.run(geom, p, seed=1, idlog=True, tables=otables, nthreads=4)
    assert _ledger_rel(r) < 1e-12
    L = r["ledger"]
    assert np.all(L[:, 4] > 0)        # every event annihilates positrons
    r1 = oracle.run(geom, p, seed=1, idlog=True, tables=otables, nthreads=1)
    assert np.array_equal(r["score"], r1["score"])
    assert np.array_equal(r["counts"], r1["counts"])
    assert np.array_equal(np.sort(r["idlog"], order="id"), np.sort(r1["idlog"], order="id"))


def test_fp64_reference_agrees_with_strict(geom, otables):
    p = W.gun(300, 1000.0)
    a = oracle.run(geom, p, seed=1, tables=otables, nthreads=4)
    b = oracle.run(geom, p, seed=1, tables=otables, nthreads=4, mode=oracle.REF_FP64)
    assert _ledger_rel(b) < 1e-12
    la = a["score"].reshape(300, 50, 2).sum(2)
    lb = b["score"].reshape(300, 50, 2).sum(2)
    diff = la - lb
    se = np.sqrt(la.var(0) / 300 + lb.var(0) / 300) + 1e-12
    assert np.all(np.abs(diff.mean(0)) <= 3 * se + 1e-9)
    tot_a, tot_b = la.sum(0), lb.sum(0)
    big = tot_a > 0.01 * tot_a.sum()
    assert np.all(np.abs(tot_a[big] - tot_b[big]) / tot_a[big] < 0.01)


@pytest.mark.parametrize("e", [0.013, 0.05, 0.3, 1.7, 25.0, 900.0, 4.2e4])
def test_transport_sees_tabulated_cross_section(otables, e):
    # with nia = 1 the physics step is 1/Sigma(E): the lookup (log, index, fraction,
    # linear interpolation) must reproduce the closed form to the interpolation error
    w = oracle.World(W.single_slab(1e9, material=0), otables, seed=1)
    tr = oracle.make_track(z=0.0, e=e, nia=1.0, slab=0)
    r = oracle.step_one(w, W.GAMMA, tr)
    assert r["lim"] == oracle.LIM_PHYS
    sig = sum(oracle.sigma(k, 0, e) for k in ("compton", "pair", "phot"))
    # linear interpolation in ln E over bins of h = ln(1e8)/256: for the E^-3 photoelectric
    # term the error is below (3h)^2/8 = 0.58%; the other terms are much flatter
    f_pe = oracle.sigma("phot", 0, e) / sig
    assert float(r["track"]["len"]) == pytest.approx(1.0 / sig, rel=0.006 * f_pe + 1e-3)
    if e > 0.02:
        tr = oracle.make_track(z=0.0, e=e, nia=1e-3, slab=0)
        r = oracle.step_one(w, W.E_MINUS, tr)
        assert r["lim"] == oracle.LIM_PHYS
        assert float(r["track"]["len"]) == pytest.approx(1e-3 / oracle.sigma("brem", 0, e), rel=2e-3)


def test_deposits_land_in_the_traversed_and_final_slabs(oworld):
    # a 15 keV electron 5 um before the lead/argon plane: the step ends on the plane
    # (geometry limit), the electron drops below the cut there; the continuous loss
    # belongs to the slab it crossed, the remainder to the slab it ended in
    z = np.float32(2.3) - np.float32(0.005)
    n_seen = 0
    for i in range(50):
        tr = oracle.make_track(z=float(z), d=(0.0, 0.0, 1.0), e=0.015, nia=1e6, slab=0, id=i)
        r = oracle.step_one(oworld, W.E_MINUS, tr)
        assert r["lim"] == oracle.LIM_Z and r["track"]["slab"] == 1
        assert r["death"] == oracle.DEATH_CUT
        assert r["slab_cont"] == 0 and r["slab_cut"] == 1
        assert r["dep_cont"] + r["cut"] == pytest.approx(0.015, rel=1e-6)
        n_seen += 1
    assert n_seen == 50


def test_interaction_lengths_carry_across_boundaries(oworld):
    # fraction of 1 MeV photons crossing one full layer (2.3 mm Pb + 5.7 mm lAr)
    # without interacting is exp(-(S_Pb 2.3 + S_Ar 5.7)) with S the total cross sections
    e, n, survived = 1.0, 20000, 0
    for i in range(n):
        tr = oracle.make_track(z=0.0, e=e, nia=-1.0, slab=0, id=i)
        while True:
            r = oracle.step_one(oworld, W.GAMMA, tr)
            if r["lim"] == oracle.LIM_PHYS:
                break
            if r["track"]["slab"] == 2:
                survived += 1
                break
            tr = np.array([r["track"]], dtype=oracle.TRACK32_DTYPE)
    s = [sum(oracle.sigma(k, m, e) for k in ("compton", "pair", "phot")) for m in (0, 1)]
    p = np.exp(-(s[0] * 2.3 + s[1] * 5.7))
    assert abs(survived / n - p) < 4 * np.sqrt(p * (1 - p) / n) + 1e-3


def test_charged_time_of_flight(oworld):
    t = 0.3
    tr = oracle.make_track(z=0.0, d=(0.0, 0.0, 1.0), e=t, nia=1e6, slab=0)
    r = oracle.step_one(oworld, W.E_MINUS, tr)
    s = float(r["track"]["len"])
    beta = np.sqrt(1.0 - (MC2 / (t + MC2)) ** 2)
    assert float(r["track"]["time"]) == pytest.approx(s / (beta * 299.792458), rel=1e-5)
