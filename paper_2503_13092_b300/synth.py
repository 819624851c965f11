"""Seeded synthetic events for the Downstream + two-track vertexing path.

This module is the only code shared by the FP64 oracle and the CUDA path: it
draws inputs (SciFi seeds, UT hits, ghost-killer weights) and the generator
truth that goes with them.  It holds none of the method's arithmetic (no
window search, fit, network evaluation or vertex solve); it only simulates the
synthetic detector world the method runs on.

The world follows the paper's description of the detector:
  * magnetic field along y, motion in B replaced by a single kink at the magnet
    point (Algorithm Design section, Eq. 1); here the kink is exact at
    z_kick = 5000 mm with a transverse kick of kappa = 1200 MeV/c (the 4 Tm
    dipole of the LHCb Detector section);
  * four UT strip layers UTaX (0 deg), UTaU (+5 deg), UTbV (-5 deg), UTbX (0 deg)
    (Fig. 2), hits grouped in 100 mm Y sectors (Algorithm Design, Dv1);
  * seeds are SciFi tracklet states at the last SciFi station (x, y, tx, ty,
    q/p, chi2) (Ghost-Killer Neural Network section);
  * mode "B" bends the track upstream of the kink with the second-order term of
    Eq. 4, its coefficient gamma taken from Eq. 3; mode "A" keeps straight lines.

Sign convention: the kink changes tx by -MP*q*kappa/p_z, the same direction as
the fringe-field curvature 2*gamma of Eq. 3 (for MP = +1 and q > 0 both bend
towards -x).  Units: mm, MeV, MeV/c; q/p in c/MeV.

Truth tracks come in opposite-charge pairs that share a vertex on the beam
axis (x = y = 0, z uniform in [0, 2000] mm), so that two-track vertexing has
true vertices to find.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, asdict

import numpy as np

LAYER_NAMES = ("UTaX", "UTaU", "UTbV", "UTbX")


@dataclass(frozen=True)
class World:
    """Constants of the synthetic detector and of its kink-model field."""

    z_layer: tuple = (2320.0, 2380.0, 2590.0, 2650.0)
    stereo_deg: tuple = (0.0, 5.0, -5.0, 0.0)
    y_min: float = -700.0
    sector_h: float = 100.0
    n_sectors: int = 14
    x_half_noise: float = 850.0      # noise hits uniform in |x| < 850 mm
    x_half_bins: float = 1000.0      # |x0| range covered by a hit-index x bin table
    z_seed: float = 9410.0           # z of the SciFi seed state
    z_kick: float = 5000.0           # exact kink position of the synthetic field
    kappa: float = 1200.0            # transverse kick, MeV/c
    mp: float = 1.0                  # magnet polarity
    z_ref: float = 2485.0            # midpoint of UTaX..UTbX, state reference plane
    gamma0: float = -1.5e-8          # Eq. 3 constants, used in mode "B"
    gamma1: float = 9.3e-3
    sigma_hit: float = 0.05          # UT hit resolution (mm)
    seed_sigma_xy: float = 0.05
    seed_sigma_t: float = 5e-5
    seed_sigma_qop_rel: float = 0.02
    p_min: float = 2000.0
    p_max: float = 100000.0
    t_max: float = 0.25
    z_vtx_max: float = 2000.0
    scifi_x_half: float = 3200.0
    scifi_y_half: float = 2400.0

    @property
    def dxdy(self):
        return tuple(math.tan(math.radians(a)) for a in self.stereo_deg)


WORLD = World()


# --------------------------------------------------------------------------------------
# truth tracks
# --------------------------------------------------------------------------------------

def _gamma(world: World, qop, mode: str):
    if mode == "A":
        return np.zeros_like(qop)
    return -world.mp * (world.gamma0 + world.gamma1 * qop)


def _propagate(world: World, zv, tx0, ty, q, p, mode):
    """Trajectory pieces of tracks leaving (0, 0, zv) with slopes (tx0, ty)."""
    pz = p / np.sqrt(1.0 + tx0 * tx0 + ty * ty)
    qop = q / p
    g = _gamma(world, qop, mode)

    def x_up(z):  # upstream of the kink: parabola (Eq. 4 form) or straight line
        dz = z - zv
        return tx0 * dz + g * dz * dz

    def y_at(z):
        return ty * (z - zv)

    tx_kink = tx0 + 2.0 * g * (world.z_kick - zv)
    tx_after = tx_kink - world.mp * q * world.kappa / pz
    x_kink = x_up(world.z_kick)
    p_after = pz * np.sqrt(1.0 + tx_after ** 2 + ty ** 2)
    x_s = x_kink + tx_after * (world.z_seed - world.z_kick)
    y_s = y_at(world.z_seed)
    return dict(x_up=x_up, y_at=y_at, tx_after=tx_after, x_s=x_s, y_s=y_s,
                qop_after=q / p_after, qop=qop, gamma=g, pz=pz)


def _accepted(world: World, traj):
    ok = np.ones_like(traj["x_s"], dtype=bool)
    y_hi = world.y_min + world.sector_h * world.n_sectors
    for z in world.z_layer:
        x = traj["x_up"](z)
        y = traj["y_at"](z)
        ok &= (np.abs(x) < world.x_half_noise) & (y > world.y_min) & (y < y_hi)
    ok &= (np.abs(traj["x_s"]) < world.scifi_x_half) & (np.abs(traj["y_s"]) < world.scifi_y_half)
    return ok


def _draw_kinematics(rng, world: World, n):
    lp = rng.uniform(math.log(world.p_min), math.log(world.p_max), n)
    tx = rng.uniform(-world.t_max, world.t_max, n)
    ty = rng.uniform(-world.t_max, world.t_max, n)
    return np.exp(lp), tx, ty


def _tracks_from_vertices(rng, world: World, zv, q, mode):
    """One accepted track per (zv, q) entry; kinematics redrawn until accepted."""
    n = zv.size
    p = np.empty(n); tx = np.empty(n); ty = np.empty(n)
    todo = np.arange(n)
    for _ in range(1000):
        if todo.size == 0:
            break
        pp, tt, uu = _draw_kinematics(rng, world, todo.size)
        tr = _propagate(world, zv[todo], tt, uu, q[todo], pp, mode)
        ok = _accepted(world, tr)
        idx = todo[ok]
        p[idx] = pp[ok]; tx[idx] = tt[ok]; ty[idx] = uu[ok]
        todo = todo[~ok]
    if todo.size:
        raise RuntimeError("track acceptance sampling did not converge")
    return p, tx, ty


def _sector_bounds(world: World, y):
    k = np.floor((y - world.y_min) / world.sector_h)
    k = np.clip(k, 0, world.n_sectors - 1)
    lo = world.y_min + k * world.sector_h
    return lo, lo + world.sector_h


# --------------------------------------------------------------------------------------
# batches
# --------------------------------------------------------------------------------------

@dataclass
class EventSpec:
    n_true: np.ndarray      # per event, even
    n_fake: np.ndarray
    n_hits: np.ndarray      # per event target total (true + noise)


def _pairs_even(n):
    return (np.asarray(n) // 2) * 2


def spec_fixed(n_events, n_true, n_fake, n_hits):
    e = n_events
    return EventSpec(np.full(e, _pairs_even(n_true)), np.full(e, n_fake), np.full(e, n_hits))


def spec_poisson(rng, n_events, mean_seeds=300, true_frac=0.4, n_hits=5000):
    ns = rng.poisson(mean_seeds, n_events)
    nt = _pairs_even(np.rint(true_frac * ns).astype(np.int64))
    return EventSpec(nt, ns - nt, np.full(n_events, n_hits))


def spec_lognormal(rng, n_events, sigma=0.77, true_frac=0.4):
    phi = rng.lognormal(0.0, sigma, n_events)
    ns = np.clip(np.rint(200 * phi), 20, 2000).astype(np.int64)
    nh = np.clip(np.rint(3000 * phi), 300, 30000).astype(np.int64)
    nt = _pairs_even(np.rint(true_frac * ns).astype(np.int64))
    return EventSpec(nt, ns - nt, nh)


def generate(spec: EventSpec, seed: int, world: World = WORLD, mode: str = "A",
             hit_eff: float = 1.0, noise_free: bool = False, kappa: float | None = None):
    """Draw a batch of events.  Returns a dict of numpy arrays (inputs + truth).

    Inputs (float32 / int32 / uint8, CSR over events):
      seed_off[E+1], seed_x, seed_y, seed_tx, seed_ty, seed_qop, seed_chi2 [S]
      hit_off[E+1], hit_x0, hit_ybeg, hit_yend [H] (f32), hit_layer [H] (u8)
    Truth (float64 / int32):
      seed_track[S] (-1 = fake), hit_track[H] (-1 = noise), trk_* per true track,
      vtx_* per true vertex (pair of opposite-charge tracks).
    `noise_free` switches off hit and seed smearing; `kappa` overrides the kick
    (0 gives a field-free world where every track is a straight line).
    """
    if kappa is not None:
        world = World(**{**asdict(world), "kappa": float(kappa)})
    rng = np.random.Generator(np.random.PCG64(seed))
    E = spec.n_true.size
    n_true = spec.n_true.astype(np.int64)
    n_fake = spec.n_fake.astype(np.int64)
    dxdy = np.array(world.dxdy)
    zl = np.array(world.z_layer)

    # true vertices and their opposite-charge daughter pairs
    n_vtx = n_true // 2
    V = int(n_vtx.sum())
    vtx_event = np.repeat(np.arange(E), n_vtx)
    vtx_z = rng.uniform(0.0, world.z_vtx_max, V)
    T = 2 * V
    trk_vertex = np.repeat(np.arange(V), 2)
    trk_event = vtx_event[trk_vertex]
    q = np.tile(np.array([1.0, -1.0]), V)
    zv = vtx_z[trk_vertex]
    p, tx0, ty = _tracks_from_vertices(rng, world, zv, q, mode)
    tr = _propagate(world, zv, tx0, ty, q, p, mode)

    # truth state at z_ref (Eq. 4 form)
    g = tr["gamma"]
    trk_state = np.stack([tr["x_up"](world.z_ref), tr["y_at"](world.z_ref),
                          tx0 + 2.0 * g * (world.z_ref - zv), ty, tr["qop"]], axis=1)

    # true hits
    hx = np.stack([tr["x_up"](z) for z in zl], axis=1)            # [T, 4]
    hy = np.stack([tr["y_at"](z) for z in zl], axis=1)
    x0 = hx - dxdy[None, :] * hy
    if not noise_free:
        x0 = x0 + rng.normal(0.0, world.sigma_hit, x0.shape)
    keep = np.ones(x0.shape, dtype=bool) if hit_eff >= 1.0 else rng.uniform(size=x0.shape) < hit_eff
    ylo, yhi = _sector_bounds(world, hy)
    th_layer = np.broadcast_to(np.arange(4), x0.shape)[keep]
    th_track = np.broadcast_to(np.arange(T)[:, None], x0.shape)[keep]
    th_x0, th_lo, th_hi = x0[keep], ylo[keep], yhi[keep]
    th_event = trk_event[th_track]

    # true seeds (smeared SciFi states)
    def smear(a, s):
        return a if noise_free else a + rng.normal(0.0, s, a.shape)
    s_x = smear(tr["x_s"], world.seed_sigma_xy)
    s_y = smear(tr["y_s"], world.seed_sigma_xy)
    s_tx = smear(tr["tx_after"], world.seed_sigma_t)
    s_ty = smear(ty, world.seed_sigma_t)
    s_qop = tr["qop_after"] * (1.0 if noise_free else (1.0 + rng.normal(0.0, world.seed_sigma_qop_rel, T)))
    s_chi2 = rng.exponential(1.0, T)

    # fake seeds: same kinematics, no UT hits
    F = int(n_fake.sum())
    f_event = np.repeat(np.arange(E), n_fake)
    f_zv = rng.uniform(0.0, world.z_vtx_max, F)
    f_q = np.where(rng.uniform(size=F) < 0.5, 1.0, -1.0)
    fp, ftx, fty = _tracks_from_vertices(rng, world, f_zv, f_q, mode)
    ftr = _propagate(world, f_zv, ftx, fty, f_q, fp, mode)
    f_x = smear(ftr["x_s"], world.seed_sigma_xy)
    f_y = smear(ftr["y_s"], world.seed_sigma_xy)
    f_tx = smear(ftr["tx_after"], world.seed_sigma_t)
    f_ty = smear(fty, world.seed_sigma_t)
    f_qop = ftr["qop_after"] * (1.0 if noise_free else (1.0 + rng.normal(0.0, world.seed_sigma_qop_rel, F)))
    f_chi2 = 3.0 * rng.exponential(1.0, F)

    # noise hits up to each event's total
    n_th = np.bincount(th_event, minlength=E)
    n_noise = np.maximum(spec.n_hits.astype(np.int64) - n_th, 0)
    N = int(n_noise.sum())
    n_event = np.repeat(np.arange(E), n_noise)
    n_layer = rng.integers(0, 4, N)
    n_xx = rng.uniform(-world.x_half_noise, world.x_half_noise, N)
    n_yy = rng.uniform(world.y_min, world.y_min + world.sector_h * world.n_sectors, N)
    n_x0 = n_xx - dxdy[n_layer] * n_yy
    n_lo, n_hi = _sector_bounds(world, n_yy)

    # assemble seeds: grouped by event, random order inside each event
    S_event = np.concatenate([trk_event, f_event])
    S_track = np.concatenate([np.arange(T), np.full(F, -1)])
    S_cols = [np.concatenate(c) for c in ((s_x, f_x), (s_y, f_y), (s_tx, f_tx), (s_ty, f_ty),
                                          (s_qop, f_qop), (s_chi2, f_chi2))]
    order = np.lexsort((rng.uniform(size=S_event.size), S_event))
    seed_off = np.zeros(E + 1, np.int32)
    seed_off[1:] = np.cumsum(np.bincount(S_event, minlength=E))

    H_event = np.concatenate([th_event, n_event])
    H_track = np.concatenate([th_track, np.full(N, -1)])
    H_layer = np.concatenate([th_layer, n_layer])
    H_x0 = np.concatenate([th_x0, n_x0])
    H_lo = np.concatenate([th_lo, n_lo])
    H_hi = np.concatenate([th_hi, n_hi])
    horder = np.lexsort((rng.uniform(size=H_event.size), H_event))
    hit_off = np.zeros(E + 1, np.int32)
    hit_off[1:] = np.cumsum(np.bincount(H_event, minlength=E))

    f32 = np.float32
    out = dict(
        n_events=E,
        seed_off=seed_off,
        seed_x=S_cols[0][order].astype(f32), seed_y=S_cols[1][order].astype(f32),
        seed_tx=S_cols[2][order].astype(f32), seed_ty=S_cols[3][order].astype(f32),
        seed_qop=S_cols[4][order].astype(f32), seed_chi2=S_cols[5][order].astype(f32),
        seed_track=S_track[order].astype(np.int32),
        hit_off=hit_off,
        hit_x0=H_x0[horder].astype(f32), hit_ybeg=H_lo[horder].astype(f32),
        hit_yend=H_hi[horder].astype(f32), hit_layer=H_layer[horder].astype(np.uint8),
        hit_track=H_track[horder].astype(np.int32),
        trk_event=trk_event.astype(np.int32), trk_q=q, trk_p=p, trk_state=trk_state,
        trk_vertex=trk_vertex.astype(np.int32), trk_gamma=g,
        vtx_event=vtx_event.astype(np.int32), vtx_z=vtx_z,
        mode=mode, world=world,
    )
    return out


def config_batch(name: str, seed: int | None = None, **kw):
    """Batches shaped like the paper's workloads (synthetic stand-ins).

    c1: one event, 50 true tracks + 150 fake seeds, ~1500 UT hits.
    c2: 1000 events, Poisson(300) seeds (40 % true), 5000 UT hits per event.
    c3: 10000 events, log-normal occupancy: seeds 20..2000, hits 300..30000.
    """
    if name == "c1":
        s = 0 if seed is None else seed
        return generate(spec_fixed(1, 50, 150, 1500), s, **kw)
    if name == "c2":
        s = 2 if seed is None else seed
        n_events = kw.pop("n_events", 1000)
        rng = np.random.Generator(np.random.PCG64(10_000 + s))
        return generate(spec_poisson(rng, n_events), s, **kw)
    if name == "c3":
        s = 3 if seed is None else seed
        n_events = kw.pop("n_events", 10000)
        rng = np.random.Generator(np.random.PCG64(10_000 + s))
        return generate(spec_lognormal(rng, n_events), s, **kw)
    raise ValueError(name)



def c5_pool(n_events: int = 4000, seed: int = 5):
    """Events of config-1 occupancy (50 true tracks + 150 fake seeds, ~1500 UT
    hits each) from which the serving workload's requests are cut."""
    return generate(spec_fixed(n_events, 50, 150, 1500), seed)


def c5_trace(n_requests: int, rate_hz: float, pool_events: int, seed: int = 5, max_events: int = 500):
    """Serving workload: request sizes uniform in 1..max_events events, Poisson
    arrivals at rate_hz (exponential gaps), each request a contiguous run of
    pool events.  Returns (sizes, first pool event, arrival time in s)."""
    rng = np.random.Generator(np.random.PCG64(20_000 + seed))
    sizes = rng.integers(1, max_events + 1, n_requests)
    arrivals = np.cumsum(rng.exponential(1.0 / rate_hz, n_requests))
    starts = rng.integers(0, pool_events - sizes + 1)
    return sizes, starts, arrivals


def slice_events(b: dict, e0: int, e1: int) -> dict:
    """Events [e0, e1) of batch b as a batch of their own (views where possible)."""
    s0, s1 = int(b["seed_off"][e0]), int(b["seed_off"][e1])
    h0, h1 = int(b["hit_off"][e0]), int(b["hit_off"][e1])
    out = dict(n_events=e1 - e0, mode=b.get("mode", "A"),
               seed_off=(b["seed_off"][e0:e1 + 1] - s0).astype(np.int32),
               hit_off=(b["hit_off"][e0:e1 + 1] - h0).astype(np.int32))
    for k in ("seed_x", "seed_y", "seed_tx", "seed_ty", "seed_qop", "seed_chi2", "seed_track"):
        if k in b:
            out[k] = b[k][s0:s1]
    for k in ("hit_x0", "hit_ybeg", "hit_yend", "hit_layer", "hit_track"):
        if k in b:
            out[k] = b[k][h0:h1]
    return out

# --------------------------------------------------------------------------------------
# ghost-killer weights (inputs to the method; fixed seed, not trained)
# --------------------------------------------------------------------------------------

def nn_weights(n_in=16, n_h1=32, n_h2=32, seed=0, out_bias=0.0):
    """Fixed-seed ghost-killer weights: Xavier-uniform from PCG64(seed), zero biases.

    Layout: row-major [out][in] per layer.  n_h2 = 0 gives the paper's single
    hidden layer network (8 -> 14 -> 1, Ghost-Killer Neural Network section).
    The input normalisation (mean, scale) maps the 16 track features to O(1).
    """
    rng = np.random.Generator(np.random.PCG64(seed))

    def xavier(fo, fi):
        a = math.sqrt(6.0 / (fi + fo))
        return rng.uniform(-a, a, (fo, fi)).astype(np.float32)

    w1 = xavier(n_h1, n_in)
    b1 = np.zeros(n_h1, np.float32)
    if n_h2 > 0:
        w2 = xavier(n_h2, n_h1)
        b2 = np.zeros(n_h2, np.float32)
        w3 = xavier(1, n_h2)[0]
    else:
        w2 = np.zeros((0, 0), np.float32)
        b2 = np.zeros(0, np.float32)
        w3 = xavier(1, n_h1)[0]
    b3 = np.float32(out_bias)
    mean = np.zeros(16, np.float32)
    # feature order: x/1e3, y/1e3, tx, ty, 1e3*qop, chi2/ndof, 1e3*qop_seed, chi2_seed,
    # 4 residual pulls, n_hits/4, |dx_bX|/W1, tx_seed, ty_seed
    scale = np.array([1.5, 1.5, 4.0, 4.0, 2.0, 0.3, 2.0, 0.5,
                      0.2, 0.2, 0.2, 0.2, 1.0, 1.0, 3.0, 4.0], np.float32)
    mean[12] = 0.875
    mean[13] = 0.5
    return dict(n_in=n_in, n_h1=n_h1, n_h2=n_h2, w1=w1, b1=b1, w2=w2, b2=b2, w3=w3.astype(np.float32),
                b3=b3, mean=mean[:n_in].copy(), scale=scale[:n_in].copy())



def line_weights(n_lines=4, n_in=16, n_h1=32, seed=100):
    """Fixed-seed trigger-line networks (Expected Physics Impact section: one
    hidden layer of 32 nodes, one output): Xavier-uniform from PCG64(seed + k),
    zero biases, identity normalisation (the 16 vertex inputs are scaled to
    O(1) by their definition).  Not trained."""
    nets = []
    for k in range(n_lines):
        w = nn_weights(n_in=n_in, n_h1=n_h1, n_h2=0, seed=seed + k)
        w["mean"] = np.zeros(n_in, np.float32)
        w["scale"] = np.ones(n_in, np.float32)
        nets.append(w)
    return nets

# --------------------------------------------------------------------------------------
# geometry + method parameters (plain numbers handed to both implementations)
# --------------------------------------------------------------------------------------

def default_config(world: World = WORLD, mode: str = "A", **overrides):
    """Geometry of the synthetic world and the method's tunable parameters.

    Window sizes follow the synthetic world's smearing: the first window
    half-width w1a + w1b*|q/p| covers three standard deviations of the seed's
    q/p smear over the 2350 mm lever arm from the magnet point to UTbX; the
    refined window w2 = 2 mm; training mode uses 100 mm / 10 mm windows with
    clone killing off (Ghost-Killer Neural Network section).
    """
    cfg = dict(
        z_layer=list(world.z_layer), dxdy=list(world.dxdy), z_seed=world.z_seed,
        zmag=[world.z_kick, 0.0, 0.0, 0.0], kappa=world.kappa, mp=world.mp,
        gamma0=world.gamma0 if mode == "B" else 0.0,
        gamma1=world.gamma1 if mode == "B" else 0.0,
        z_ref=world.z_ref, sigma_hit=world.sigma_hit, sigma_mag=1.0,
        y_min=world.y_min, sector_h=world.sector_h, n_sectors=world.n_sectors,
        x_half_bins=world.x_half_bins,
        w1a=3.0, w1b=1.7e5, w2=2.0, dy_tol=2.0, k1=10,
        first_window_origin=0, pick_chi2=0, clone_kill=1, training=0,
        nn_threshold=0.5, doca_max=2.0, nr_tol=1e-6, nr_max_iter=10,
        variant=0, dv1_dtx_max=0.8, dv1_w_tri=1.0,
    )
    for k, v in overrides.items():
        if k not in cfg:
            raise KeyError(k)
        cfg[k] = v
    return cfg
