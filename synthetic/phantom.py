"""Seeded head-and-neck-shaped phantoms and random sparse problems.

The paper plans on TCIA patients with matRad pencil-beam dose (Sec. 2.3,
Table 1); neither is available, so problems are synthesised here with the
paper's shapes: m voxels, n proton spots on a lateral grid with energy layers,
N uncertainty scenarios (setup shifts of the isocentre and range scalings),
dose entries truncated relative to the matrix maximum, rows = voxels.

Dose model (a stand-in chosen for this build, not matRad):
    dose(voxel, spot) = G(r_perp; sigma) * B(depth; R)
    G(r) = exp(-r^2 / (2 sigma^2))                         lateral Gaussian
    B(d; R) = 0.25 + 0.75 exp(-(d-R)^2/(2 sR^2))  for d <= R   (entrance plateau)
            = exp(-(d-R)^2/(2 sR^2))              for d >  R   (distal fall-off)
    sR = 0.012 R + 1 mm
depth = distance from the body surface along the beam direction.  A setup
shift evaluates the dose at (voxel + shift); a range scaling multiplies depth
by (1 + kappa).  Everything is float64 until the final float32 cast.

Nothing in this module solves the optimisation problem.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

# ----------------------------------------------------------------------------
# problem container
# ----------------------------------------------------------------------------


@dataclass
class Problem:
    """A robust planning problem in the layout the C-ABI takes.

    row_ptr[s] int32[m+1], col_idx[s] int32[nnz_s] (sorted within each row),
    val[s] float32[nnz_s] (>= 0): dose-influence matrix A_s of scenario s,
    rows = voxels, columns = spots.  voxel_w float64[m] (>= 0), presc
    float64[m] (>= 0), scen_weight float64[N] or None (= all ones), lb/ub
    float64[n].
    """

    m: int
    n: int
    N: int
    row_ptr: list
    col_idx: list
    val: list
    voxel_w: np.ndarray
    presc: np.ndarray
    scen_weight: np.ndarray | None
    lb: np.ndarray
    ub: np.ndarray
    labels: np.ndarray | None = None
    meta: dict = field(default_factory=dict)

    def nnz(self) -> list[int]:
        return [int(v.size) for v in self.val]

    def csr(self, s: int) -> sp.csr_matrix:
        """Scenario s as a scipy CSR matrix (float64 copy of the float32 values)."""
        return sp.csr_matrix(
            (self.val[s].astype(np.float64), self.col_idx[s], self.row_ptr[s]),
            shape=(self.m, self.n),
        )

    def matrix_bytes(self, value_bytes: int = 4, index_bytes: int = 4) -> int:
        return sum(v.size * (value_bytes + index_bytes) for v in self.val)

    def subset_scenarios(self, idx) -> "Problem":
        idx = list(idx)
        return Problem(
            m=self.m, n=self.n, N=len(idx),
            row_ptr=[self.row_ptr[i] for i in idx],
            col_idx=[self.col_idx[i] for i in idx],
            val=[self.val[i] for i in idx],
            voxel_w=self.voxel_w, presc=self.presc,
            scen_weight=None if self.scen_weight is None else self.scen_weight[idx],
            lb=self.lb, ub=self.ub, labels=self.labels, meta=dict(self.meta),
        )


# ----------------------------------------------------------------------------
# scenario sets
# ----------------------------------------------------------------------------


def scenario_set_13(shift_mm: float = 3.0, range_frac: float = 0.035):
    """Nominal, six +-shift axis shifts, and +-range x {no shift, +z, -z}: 13.

    Returns a list of (dx, dy, dz, kappa); depth is multiplied by (1 + kappa).
    """
    s, k = shift_mm, range_frac
    out = [(0.0, 0.0, 0.0, 0.0)]
    for ax in range(3):
        for sg in (+1.0, -1.0):
            d = [0.0, 0.0, 0.0]
            d[ax] = sg * s
            out.append((d[0], d[1], d[2], 0.0))
    for dz in (0.0, +s, -s):
        for kk in (+k, -k):
            out.append((0.0, 0.0, dz, kk))
    assert len(out) == 13
    return out


def scenario_set_49(shift_mm: float = 3.0, range_frac: float = 0.035):
    """27 lattice shifts at nominal range, plus +-range at 11 positions: 49.

    The 11 positions: the centre, the 6 axis shifts and the 4 in-plane (x, y)
    diagonals at z = 0.
    """
    s, k = shift_mm, range_frac
    out = []
    for dz in (-s, 0.0, s):
        for dy in (-s, 0.0, s):
            for dx in (-s, 0.0, s):
                out.append((dx, dy, dz, 0.0))
    pos = [(0.0, 0.0, 0.0)]
    for ax in range(3):
        for sg in (+1.0, -1.0):
            d = [0.0, 0.0, 0.0]
            d[ax] = sg * s
            pos.append(tuple(d))
    for sx in (+1.0, -1.0):
        for sy in (+1.0, -1.0):
            pos.append((sx * s, sy * s, 0.0))
    for p in pos:
        for kk in (+k, -k):
            out.append((p[0], p[1], p[2], kk))
    assert len(out) == 49
    return out


# ----------------------------------------------------------------------------
# geometry
# ----------------------------------------------------------------------------


class _Box:
    def __init__(self, half):
        self.half = np.asarray(half, dtype=np.float64)

    def inside(self, Q):
        return np.all(np.abs(Q) <= self.half + 1e-9, axis=1)

    def depth(self, Q, d):
        """Distance from Q back along -d to the box surface (nan outside)."""
        t = np.full(Q.shape[0], np.inf)
        for k in range(3):
            if d[k] > 1e-12:
                t = np.minimum(t, (Q[:, k] + self.half[k]) / d[k])
            elif d[k] < -1e-12:
                t = np.minimum(t, (self.half[k] - Q[:, k]) / (-d[k]))
        t[~self.inside(Q)] = np.nan
        return t


class _Ellipsoid:
    def __init__(self, center, semi):
        self.c = np.asarray(center, dtype=np.float64)
        self.s = np.asarray(semi, dtype=np.float64)

    def inside(self, Q):
        return np.sum(((Q - self.c) / self.s) ** 2, axis=1) <= 1.0

    def depth(self, Q, d):
        X = (Q - self.c) / self.s
        D = np.asarray(d, dtype=np.float64) / self.s
        a = D @ D
        b = X @ D
        c = np.sum(X * X, axis=1) - 1.0
        disc = b * b - a * c
        t = (b + np.sqrt(np.maximum(disc, 0.0))) / a
        t[c > 0.0] = np.nan
        return t

    def ray_span(self, origin, d):
        """Parameters t_in <= t_out where origin + t d crosses the surface, or None."""
        X = (np.asarray(origin) - self.c) / self.s
        D = np.asarray(d) / self.s
        a = D @ D
        b = X @ D
        c = X @ X - 1.0
        disc = b * b - a * c
        if disc <= 0:
            return None
        r = math.sqrt(disc)
        return (-b - r) / a, (-b + r) / a


def _beam_frame(angle_deg):
    th = math.radians(angle_deg)
    d = np.array([math.cos(th), math.sin(th), 0.0])
    e1 = np.array([-math.sin(th), math.cos(th), 0.0])
    e2 = np.array([0.0, 0.0, 1.0])
    return d, e1, e2


def _grid_centers(shape, h):
    nx, ny, nz = shape
    xs = (np.arange(nx) + 0.5 - nx / 2.0) * h
    ys = (np.arange(ny) + 0.5 - ny / 2.0) * h
    zs = (np.arange(nz) + 0.5 - nz / 2.0) * h
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")  # x fastest
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)


def _bragg(dep, R):
    sR = 0.012 * R + 1.0
    x = dep - R
    g = np.exp(-(x * x) / (2.0 * sR * sR))
    return np.where(x <= 0.0, 0.25 + 0.75 * g, g)


# ----------------------------------------------------------------------------
# dose-influence matrices
# ----------------------------------------------------------------------------


@dataclass
class _Beam:
    angle: float
    iso: np.ndarray
    spacing: float            # lateral grid spacing (mm)
    lat_ij: np.ndarray        # int [L, 2] lateral grid indices (u = i*spacing, v = j*spacing)
    lat_start: np.ndarray     # int [L] first spot id of each lateral position
    lat_count: np.ndarray     # int [L] spots (energy layers) at each lateral position
    R: np.ndarray             # float [n_beam_spots] ranges (mm), spot order


def _beam_entries(P, body, beam, spot_offset, shift, kappa, sigma):
    """(row, col, value) of one beam in one scenario, before truncation."""
    d, e1, e2 = _beam_frame(beam.angle)
    Q = P + np.asarray(shift, dtype=np.float64)
    dep = body.depth(Q, d)
    ok = np.isfinite(dep)
    vox = np.nonzero(ok)[0]
    Qv = Q[vox] - beam.iso
    dep = dep[vox] * (1.0 + kappa)
    u = Qv @ e1
    v = Qv @ e2
    rcut = 4.0 * sigma
    s = beam.spacing
    K = int(math.ceil(rcut / s)) + 1
    iu0 = np.rint(u / s).astype(np.int64)
    iv0 = np.rint(v / s).astype(np.int64)
    # lateral-position lookup table over the grid's index box
    li = beam.lat_ij
    imin, jmin = li.min(axis=0) - K - 1
    imax, jmax = li.max(axis=0) + K + 1
    table = np.full((imax - imin + 1, jmax - jmin + 1), -1, dtype=np.int64)
    table[li[:, 0] - imin, li[:, 1] - jmin] = np.arange(li.shape[0])
    # deepest reach of each lateral position (max range + 4 sR)
    Rmax = np.array([beam.R[a:a + c].max() for a, c in zip(beam.lat_start, beam.lat_count)])
    reach = Rmax + 4.0 * (0.012 * Rmax + 1.0)
    rows, lats, gs, deps = [], [], [], []
    for du in range(-K, K + 1):
        for dv in range(-K, K + 1):
            iu = iu0 + du
            iv = iv0 + dv
            inb = (iu >= imin) & (iu <= imax) & (iv >= jmin) & (iv <= jmax)
            lp = np.full(iu.shape, -1, dtype=np.int64)
            lp[inb] = table[iu[inb] - imin, iv[inb] - jmin]
            r2 = (u - iu * s) ** 2 + (v - iv * s) ** 2
            keep = (lp >= 0) & (r2 <= rcut * rcut)
            idx = np.nonzero(keep)[0]
            if idx.size == 0:
                continue
            keep2 = dep[idx] <= reach[lp[idx]]
            idx = idx[keep2]
            rows.append(vox[idx])
            lats.append(lp[idx])
            gs.append(np.exp(-r2[idx] / (2.0 * sigma * sigma)))
            deps.append(dep[idx])
    if not rows:
        z = np.zeros(0)
        return z.astype(np.int64), z.astype(np.int64), z
    rows = np.concatenate(rows)
    lats = np.concatenate(lats)
    gs = np.concatenate(gs)
    deps = np.concatenate(deps)
    rep = beam.lat_count[lats]
    tot = int(rep.sum())
    first = np.repeat(beam.lat_start[lats], rep)
    within = np.arange(tot) - np.repeat(np.cumsum(rep) - rep, rep)
    spot = first + within
    dep_e = np.repeat(deps, rep)
    R_e = beam.R[spot]
    sR = 0.012 * R_e + 1.0
    near = dep_e <= R_e + 4.0 * sR
    val = np.repeat(gs, rep)[near] * _bragg(dep_e[near], R_e[near])
    return np.repeat(rows, rep)[near], (spot[near] + spot_offset), val


def _scenario_matrix(args):
    P, body, beams, offsets, shift, kappa, sigma, m, n = args
    R, C, V = [], [], []
    for beam, off in zip(beams, offsets):
        r, c, v = _beam_entries(P, body, beam, off, shift, kappa, sigma)
        R.append(r)
        C.append(c)
        V.append(v)
    r = np.concatenate(R)
    c = np.concatenate(C)
    v = np.concatenate(V)
    return r, c, v


def _to_csr(r, c, v, m, n):
    M = sp.coo_matrix((v, (r, c)), shape=(m, n)).tocsr()
    M.sum_duplicates()
    M.sort_indices()
    return M


def _build_matrices(P, body, beams, scenarios, sigma, m, n, tau, nnz_per_col,
                    target_mask, d_pres, workers):
    offsets = np.cumsum([0] + [b.R.size for b in beams[:-1]])
    jobs = [(P, body, beams, offsets, sc[:3], sc[3], sigma, m, n) for sc in scenarios]
    if workers and workers > 1 and len(jobs) > 1:
        import multiprocessing as mp
        ctx = mp.get_context("spawn")
        with ctx.Pool(min(workers, len(jobs))) as pool:
            raw = pool.map(_scenario_matrix, jobs)
    else:
        raw = [_scenario_matrix(j) for j in jobs]
    # truncation factor: given, or tuned on the nominal scenario (index 0)
    if tau is None:
        v0 = raw[0][2]
        want = int(nnz_per_col * n)
        if want >= v0.size:
            tau = 0.0
        else:
            kth = np.partition(v0, v0.size - want)[v0.size - want]
            tau = float(kth / v0.max())
    mats = []
    for (r, c, v) in raw:
        thr = tau * v.max() if v.size else 0.0
        keep = v >= thr
        mats.append(_to_csr(r[keep], c[keep], v[keep], m, n))
    # global scale: x = 1 gives a mean nominal target dose of d_pres / 3
    tdose = mats[0] @ np.ones(n)
    scale = (d_pres / 3.0) / float(tdose[target_mask].mean())
    out_rp, out_ci, out_v = [], [], []
    for M in mats:
        out_rp.append(M.indptr.astype(np.int32))
        out_ci.append(M.indices.astype(np.int32))
        out_v.append((M.data * scale).astype(np.float32))
    return out_rp, out_ci, out_v, tau, scale


# ----------------------------------------------------------------------------
# configurations
# ----------------------------------------------------------------------------


def _label_voxels(P, body, target, oars):
    """-1 outside body, 0 body, 1 target, 2.. OARs (target has priority)."""
    lab = np.full(P.shape[0], -1, dtype=np.int8)
    lab[body.inside(P)] = 0
    for k, o in enumerate(oars):
        lab[(lab >= 0) & o.inside(P)] = 2 + k
    lab[(lab >= 0) & target.inside(P)] = 1
    return lab


def _lateral_grid_square(half_count):
    ii, jj = np.meshgrid(np.arange(-half_count, half_count + 1),
                         np.arange(-half_count, half_count + 1), indexing="ij")
    return np.stack([ii.ravel(), jj.ravel()], axis=1)


def config_tiny_plain(seed: int = 0, scenarios=None, workers: int = 0) -> Problem:
    """20x20x20 grid at 2 mm; target sphere r = 6 mm (70 Gy, w 100); OAR sphere
    r = 4 mm 5 mm from the target edge (0 Gy, w 10); body = rest (0 Gy, w 1);
    200 spots from beams at 0 and 90 degrees (5x5 lateral grid at 3 mm x 4
    energy layers, ranges uniform over the target's depth span +- 3 mm);
    13 scenarios; entries below 1e-3 * max dropped; bounds [0, 10].
    """
    rng = np.random.default_rng(seed)
    shape, h = (20, 20, 20), 2.0
    Pall = _grid_centers(shape, h)
    body = _Box([20.0, 20.0, 20.0])
    target = _Ellipsoid([0.0, 0.0, 0.0], [6.0, 6.0, 6.0])
    oar = _Ellipsoid([15.0, 0.0, 0.0], [4.0, 4.0, 4.0])
    lab_all = _label_voxels(Pall, body, target, [oar])
    keep = lab_all >= 0
    P = Pall[keep]
    lab = lab_all[keep]
    m = P.shape[0]
    beams = []
    for ang in (0.0, 90.0):
        d, _, _ = _beam_frame(ang)
        iso = np.zeros(3)
        d_iso = float(body.depth(iso[None, :], d)[0])
        lo, hi = d_iso - 6.0 - 3.0, d_iso + 6.0 + 3.0
        lat = _lateral_grid_square(2)          # 5 x 5
        L = lat.shape[0]
        cnt = np.full(L, 4, dtype=np.int64)
        start = np.arange(L, dtype=np.int64) * 4
        R = rng.uniform(lo, hi, size=4 * L)
        beams.append(_Beam(ang, iso, 3.0, lat, start, cnt, R))
    n = sum(b.R.size for b in beams)
    scen = scenarios if scenarios is not None else scenario_set_13()
    w = np.where(lab == 1, 100.0, np.where(lab >= 2, 10.0, 1.0))
    p = np.where(lab == 1, 70.0, 0.0)
    rp, ci, va, tau, scale = _build_matrices(
        P, body, beams, scen, 3.0, m, n, 1e-3, None, lab == 1, 70.0, workers)
    return Problem(
        m=m, n=n, N=len(scen), row_ptr=rp, col_idx=ci, val=va,
        voxel_w=w.astype(np.float64), presc=p.astype(np.float64), scen_weight=None,
        lb=np.zeros(n), ub=np.full(n, 10.0), labels=lab,
        meta=dict(name="tiny-plain 20^3 grid, 200 spots, 13 scenarios", seed=seed,
                  tau=tau, scale=scale, scenarios=scen),
    )


def _beam_spots_for_target(body, target, ang, spacing, n_spots, margin, rng):
    """Lateral grid points whose ray crosses the (margin-expanded) target, with
    energy layers apportioned to the crossed depth span; exactly n_spots."""
    d, e1, e2 = _beam_frame(ang)
    iso = target.c.copy()
    tgt = _Ellipsoid(target.c, target.s + margin)
    rmax = float(np.max(tgt.s))
    hc = int(math.ceil(rmax / spacing)) + 1
    lat_all = _lateral_grid_square(hc)
    lat, spans = [], []
    for (i, j) in lat_all:
        o = iso + i * spacing * e1 + j * spacing * e2
        sp_ = tgt.ray_span(o - 500.0 * d, d)
        if sp_ is None:
            continue
        p_in = o - 500.0 * d + sp_[0] * d
        p_out = o - 500.0 * d + sp_[1] * d
        d_in = float(body.depth(p_in[None, :], d)[0])
        d_out = float(body.depth(p_out[None, :], d)[0])
        if not (np.isfinite(d_in) and np.isfinite(d_out)):
            continue
        lat.append((i, j))
        spans.append((d_in, d_out))
    lat = np.asarray(lat, dtype=np.int64)
    spans = np.asarray(spans)
    length = spans[:, 1] - spans[:, 0] + 2.0
    # largest-remainder apportionment, at least one layer per position
    L = lat.shape[0]
    if n_spots < L:
        raise ValueError("fewer spots than lateral positions")
    quota = length / length.sum() * (n_spots - L)
    cnt = 1 + np.floor(quota).astype(np.int64)
    rem = n_spots - int(cnt.sum())
    order = np.argsort(-(quota - np.floor(quota)), kind="stable")
    cnt[order[:rem]] += 1
    start = np.concatenate([[0], np.cumsum(cnt)[:-1]]).astype(np.int64)
    R = np.empty(n_spots)
    for k in range(L):
        a, b = spans[k]
        c = cnt[k]
        base = a + (np.arange(c) + 0.5) / c * (b - a)
        R[start[k]:start[k] + c] = base + rng.uniform(-1.0, 1.0, size=c)
    return _Beam(ang, iso, spacing, lat, start, cnt, R)


def config_realistic(seed: int = 0, n_spots: int = 5000, nnz_per_col: float = 2000.0,
                     scenarios=None, workers: int = 8, grid=(128, 128, 96), h: float = 2.5,
                     beams_deg=(0.0, 120.0, 240.0), scale: float = 1.0) -> Problem:
    """128x128x96 grid at 2.5 mm; body ellipsoid of ~300k voxels; ellipsoidal
    target (70 Gy, w 100) and three OAR ellipsoids (0 Gy, w 10); body (0 Gy,
    w 1); n_spots from 3 beams on a 5 mm lateral grid; 13 scenarios; the
    truncation factor is tuned on the nominal scenario to nnz_per_col entries
    per spot column; bounds [0, 10].  `scale` multiplies every length of the
    geometry and the grid extent (voxel size fixed): about 300k * scale^3 voxels.
    """
    rng = np.random.default_rng(seed)
    if scale != 1.0:
        grid = tuple(max(8, int(round(g * scale))) for g in grid)
    Pall = _grid_centers(grid, h)
    sc = float(scale)
    body = _Ellipsoid([0.0, 0.0, 0.0], [90.0 * sc, 105.0 * sc, 118.0 * sc])
    target = _Ellipsoid([10.0 * sc, 5.0 * sc, 0.0], [30.0 * sc, 28.0 * sc, 32.0 * sc])
    oars = [
        _Ellipsoid([-42.0 * sc, 0.0, 10.0 * sc], [12.0 * sc, 15.0 * sc, 20.0 * sc]),
        _Ellipsoid([35.0 * sc, 45.0 * sc, -10.0 * sc], [10.0 * sc, 12.0 * sc, 15.0 * sc]),
        _Ellipsoid([0.0, -55.0 * sc, 0.0], [8.0 * sc, 8.0 * sc, 60.0 * sc]),
    ]
    lab_all = _label_voxels(Pall, body, target, oars)
    keep = lab_all >= 0
    P = Pall[keep]
    lab = lab_all[keep]
    m = P.shape[0]
    nb = len(beams_deg)
    per = [n_spots // nb + (1 if k < n_spots % nb else 0) for k in range(nb)]
    beams = [_beam_spots_for_target(body, target, a, 5.0, c, 1.0, rng)
             for a, c in zip(beams_deg, per)]
    n = sum(b.R.size for b in beams)
    scen = scenarios if scenarios is not None else scenario_set_13()
    w = np.where(lab == 1, 100.0, np.where(lab >= 2, 10.0, 1.0))
    p = np.where(lab == 1, 70.0, 0.0)
    rp, ci, va, tau, scale = _build_matrices(
        P, body, beams, scen, 3.0, m, n, None, nnz_per_col, lab == 1, 70.0, workers)
    return Problem(
        m=m, n=n, N=len(scen), row_ptr=rp, col_idx=ci, val=va,
        voxel_w=w.astype(np.float64), presc=p.astype(np.float64), scen_weight=None,
        lb=np.zeros(n), ub=np.full(n, 10.0), labels=lab,
        meta=dict(name=f"realistic {grid} grid, {n} spots, {len(scen)} scenarios",
                  seed=seed, tau=tau, scale=scale, scenarios=scen),
    )


def random_problem(seed: int, m: int, n: int, N: int, mean_row: float = 6.0,
                   empty_frac: float = 0.1, long_rows: int = 2, lb=0.0, ub=10.0,
                   zero_w_frac: float = 0.0, scen_weight: bool = False,
                   presc_level: float = 70.0) -> Problem:
    """Random nonnegative CSR problem with ragged rows for kernel tests.

    Row lengths are Poisson(mean_row) clipped to [1, n]; a fraction of rows is
    empty, `long_rows` rows are dense (all n columns) and at least one row has
    exactly one entry.  Columns are sorted within rows.  About a quarter of the
    voxels are 'target' voxels with prescription presc_level.
    """
    rng = np.random.default_rng(seed)
    rps, cis, vas = [], [], []
    target = rng.random(m) < 0.25
    for s in range(N):
        lens = np.clip(rng.poisson(mean_row, size=m), 1, n)
        lens[rng.random(m) < empty_frac] = 0
        if m > 0:
            lens[rng.integers(0, m)] = 1
        for r in rng.integers(0, m, size=min(long_rows, m)) if m > 0 else []:
            lens[r] = n
        rp = np.zeros(m + 1, dtype=np.int64)
        rp[1:] = np.cumsum(lens)
        ci = np.empty(int(rp[-1]), dtype=np.int32)
        for i in range(m):
            k = int(lens[i])
            if k:
                ci[rp[i]:rp[i + 1]] = np.sort(rng.choice(n, size=k, replace=False))
        va = rng.uniform(0.05, 1.0, size=ci.size).astype(np.float32)
        rps.append(rp.astype(np.int32))
        cis.append(ci)
        vas.append(va)
    w = rng.uniform(0.5, 2.0, size=m)
    w[target] *= 20.0
    if zero_w_frac > 0:
        w[rng.random(m) < zero_w_frac] = 0.0
    p = np.where(target, presc_level, 0.0)
    sw = rng.uniform(0.2, 1.0, size=N) if scen_weight else None
    return Problem(
        m=m, n=n, N=N, row_ptr=rps, col_idx=cis, val=vas, voxel_w=w, presc=p,
        scen_weight=sw, lb=np.full(n, float(lb)), ub=np.full(n, float(ub)),
        labels=target.astype(np.int8), meta=dict(name="random", seed=seed),
    )


def from_dense(A_list, w, p, lb, ub, scen_weight=None, name="dense") -> Problem:
    """Build a Problem from dense per-scenario matrices (small hand-made cases)."""
    A_list = [np.atleast_2d(np.asarray(A, dtype=np.float64)) for A in A_list]
    m, n = A_list[0].shape
    rps, cis, vas = [], [], []
    for A in A_list:
        M = sp.csr_matrix(A)
        M.eliminate_zeros()
        M.sort_indices()
        rps.append(M.indptr.astype(np.int32))
        cis.append(M.indices.astype(np.int32))
        vas.append(M.data.astype(np.float32))
    return Problem(
        m=m, n=n, N=len(A_list), row_ptr=rps, col_idx=cis, val=vas,
        voxel_w=np.asarray(w, dtype=np.float64).reshape(m),
        presc=np.asarray(p, dtype=np.float64).reshape(m),
        scen_weight=None if scen_weight is None else np.asarray(scen_weight, dtype=np.float64),
        lb=np.broadcast_to(np.asarray(lb, dtype=np.float64), (n,)).copy(),
        ub=np.broadcast_to(np.asarray(ub, dtype=np.float64), (n,)).copy(),
        meta=dict(name=name),
    )


# ---------------------------------------------------------------------------
# objective-weight sweeps (inputs of the learned warm start)
# ---------------------------------------------------------------------------
N_WEIGHT_SLOTS = 8


def reweighted(prob: Problem, struct_w, d_pres: float, target_label: int = 1) -> Problem:
    """The same geometry and matrices with new objective weights: every voxel
    gets the weight of its structure slot (slot = label: 0 body, 1 target,
    2.. organs at risk), the target the prescription d_pres, other voxels 0."""
    from copy import copy
    lab = np.asarray(prob.labels)
    sw = np.asarray(struct_w, dtype=np.float64)
    out = copy(prob)
    out.voxel_w = sw[np.clip(lab, 0, sw.size - 1)].astype(np.float64)
    out.presc = np.where(lab == target_label, float(d_pres), 0.0).astype(np.float64)
    out.meta = dict(prob.meta, struct_w=sw.tolist(), d_pres=float(d_pres))
    return out


def sample_weights(rng, labels, w_range=(0.1, 100.0), d_range=(60.0, 75.0)):
    """Seeded draw of structure weights (log-uniform, one per structure present;
    unused slots 0) and a prescription (uniform)."""
    present = np.unique(np.asarray(labels))
    sw = np.zeros(N_WEIGHT_SLOTS)
    lo, hi = np.log10(w_range[0]), np.log10(w_range[1])
    for k in present:
        if 0 <= k < N_WEIGHT_SLOTS:
            sw[k] = 10.0 ** rng.uniform(lo, hi)
    return sw, float(rng.uniform(*d_range))


# ---------------------------------------------------------------------------
# several plans at once (the batched form)
# ---------------------------------------------------------------------------
def block_diagonal(problems) -> Problem:
    """Several independent problems with the same number of scenarios as one:
    rows (voxels) and columns (spots) are stacked, scenario s of the result is
    blockdiag(A_s of each problem).  The objective is the sum of the problems'
    objectives and the box is the product of their boxes, so the optimum is
    the problems' optima side by side.  meta["blocks"] = [(row0, m, col0, n)]."""
    N = problems[0].N
    assert all(p.N == N for p in problems)
    rps, cis, vas = [], [], []
    for s in range(N):
        rp_parts, ci_parts, va_parts = [], [], []
        nnz0, col0 = 0, 0
        for p in problems:
            rp = np.asarray(p.row_ptr[s], dtype=np.int64)
            rp_parts.append(rp[:-1] + nnz0)
            ci_parts.append(np.asarray(p.col_idx[s], dtype=np.int64) + col0)
            va_parts.append(np.asarray(p.val[s], dtype=np.float32))
            nnz0 += int(rp[-1])
            col0 += p.n
        rp_all = np.concatenate(rp_parts + [np.array([nnz0], dtype=np.int64)])
        assert nnz0 < 2 ** 31
        rps.append(rp_all.astype(np.int32))
        cis.append(np.concatenate(ci_parts).astype(np.int32))
        vas.append(np.concatenate(va_parts))
    blocks, r0, c0 = [], 0, 0
    for p in problems:
        blocks.append((r0, p.m, c0, p.n))
        r0 += p.m
        c0 += p.n
    sw = problems[0].scen_weight
    labels = None if any(p.labels is None for p in problems) else np.concatenate([p.labels for p in problems])
    return Problem(
        m=r0, n=c0, N=N, row_ptr=rps, col_idx=cis, val=vas,
        voxel_w=np.concatenate([p.voxel_w for p in problems]),
        presc=np.concatenate([p.presc for p in problems]), scen_weight=sw,
        lb=np.concatenate([p.lb for p in problems]), ub=np.concatenate([p.ub for p in problems]),
        labels=labels, meta=dict(name=f"{len(problems)} plans block-diagonal", blocks=blocks))


BATCH_SIZES = ((100_000, 2000), (170_000, 3000), (230_000, 4000), (300_000, 5000))
# eight small plans of uneven size over the 13-scenario set: each alone is too
# small to fill the GPU, so one launch over all of them has room to gain
BATCH_SIZES_SMALL = ((12_000, 250), (18_000, 350), (24_000, 450), (30_000, 550),
                     (36_000, 650), (42_000, 750), (48_000, 850), (54_000, 950))


def config_batch(seed: int = 0, workers: int = 8, nnz_per_col: float = 1700.0, scenarios=None,
                 sizes=BATCH_SIZES):
    """Plans of uneven size (voxels, spots), by default four (100k/2k,
    170k/3k, 230k/4k, 300k/5k) over the 49-scenario set; realistic geometry
    scaled to each voxel count, about nnz_per_col entries per spot column.
    Returns the list."""
    scen = scenarios if scenarios is not None else scenario_set_49()
    out = []
    for k, (m, n) in enumerate(sizes):
        out.append(config_realistic(seed + 101 * k, n_spots=n, nnz_per_col=nnz_per_col, scenarios=scen,
                                    workers=workers, scale=(m / 299_088.0) ** (1.0 / 3.0)))
    return out
