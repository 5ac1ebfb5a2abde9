"""Seeded synthetic catalogs and bin edges for angular pair counting.

This module produces *inputs* only.  It holds none of the pair-counting
arithmetic: no dot products between catalog points, no angle binning and no
estimator.  Both the CPU oracle (``oracle/``) and the CUDA library consume
exactly the arrays it returns.

The paper measures on the MICE galaxy catalogs (Section 4), which are not
available here.  The generators below stand in for them with the shapes the
benchmark workloads describe: an octant, a full sphere or a spherical cap
footprint; randoms uniform on the sphere within the footprint; data with a
fraction of points in Gaussian clusters on the tangent plane and the rest as
uniform background.

Coordinates are produced as float64 right ascension / declination in degrees
and converted once to float64 unit vectors

    x = cos(dec) cos(ra),  y = cos(dec) sin(ra),  z = sin(dec)

(degrees to radians by multiplying with pi/180).  The catalogs are returned as
C-contiguous ``(n, 3)`` float64 arrays.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

DEG = math.pi / 180.0

# Independent child streams of one SeedSequence, in this fixed order.
_STREAMS = ("centres", "memberships", "offsets", "background", "randoms", "patches", "jobs")


def _rngs(seed: int) -> dict[str, np.random.Generator]:
    children = np.random.SeedSequence(seed).spawn(len(_STREAMS))
    return {name: np.random.Generator(np.random.PCG64(s)) for name, s in zip(_STREAMS, children)}


def radec_to_xyz(ra_deg: np.ndarray, dec_deg: np.ndarray) -> np.ndarray:
    """float64 RA/Dec in degrees -> (n, 3) float64 unit vectors."""
    ra = np.asarray(ra_deg, dtype=np.float64) * DEG
    dec = np.asarray(dec_deg, dtype=np.float64) * DEG
    cd = np.cos(dec)
    out = np.empty((ra.shape[0], 3), dtype=np.float64)
    out[:, 0] = cd * np.cos(ra)
    out[:, 1] = cd * np.sin(ra)
    out[:, 2] = np.sin(dec)
    return out


def _xyz_to_radec(v: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    ra = np.degrees(np.arctan2(v[:, 1], v[:, 0])) % 360.0
    dec = np.degrees(np.arcsin(np.clip(v[:, 2], -1.0, 1.0)))
    return ra, dec


# --------------------------------------------------------------------------- footprints
@dataclasses.dataclass(frozen=True)
class Footprint:
    """A sky region: ``octant`` (RA, Dec in [0, 90) deg), ``sphere``, or ``cap``
    (centre ``ra0``/``dec0`` in degrees, radius ``radius`` in degrees)."""

    kind: str = "octant"
    ra0: float = 0.0
    dec0: float = 0.0
    radius: float = 0.0

    def uniform(self, rng: np.random.Generator, n: int) -> tuple[np.ndarray, np.ndarray]:
        """n points uniform on the sphere within the footprint (RA, Dec in degrees)."""
        if self.kind == "octant":
            ra = rng.uniform(0.0, 90.0, n)
            dec = np.degrees(np.arcsin(rng.uniform(0.0, 1.0, n)))
            return ra, dec
        if self.kind == "sphere":
            ra = rng.uniform(0.0, 360.0, n)
            dec = np.degrees(np.arcsin(rng.uniform(-1.0, 1.0, n)))
            return ra, dec
        if self.kind == "cap":
            cosr = math.cos(self.radius * DEG)
            cs = rng.uniform(cosr, 1.0, n)          # cos(separation from the centre)
            pa = rng.uniform(0.0, 2.0 * math.pi, n)  # position angle
            return self._from_cap(cs, pa)
        raise ValueError(f"unknown footprint {self.kind!r}")

    def _from_cap(self, cs: np.ndarray, pa: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
        c = radec_to_xyz(np.array([self.ra0]), np.array([self.dec0]))[0]
        e_a, e_d = _tangent_basis(c[None, :])
        sn = np.sqrt(np.maximum(0.0, 1.0 - cs * cs))
        v = (cs[:, None] * c[None, :]
             + (sn * np.cos(pa))[:, None] * e_a
             + (sn * np.sin(pa))[:, None] * e_d)
        v /= np.linalg.norm(v, axis=1)[:, None]
        return _xyz_to_radec(v)

    def contains(self, ra: np.ndarray, dec: np.ndarray) -> np.ndarray:
        if self.kind == "octant":
            return (ra >= 0.0) & (ra < 90.0) & (dec >= 0.0) & (dec < 90.0)
        if self.kind == "sphere":
            return np.ones(ra.shape, dtype=bool)
        if self.kind == "cap":
            c = radec_to_xyz(np.array([self.ra0]), np.array([self.dec0]))[0]
            v = radec_to_xyz(ra, dec)
            return v @ c >= math.cos(self.radius * DEG)
        raise ValueError(self.kind)


def _tangent_basis(c: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Unit vectors along increasing RA and Dec at the unit vectors ``c``."""
    ra = np.arctan2(c[:, 1], c[:, 0])
    dec = np.arcsin(np.clip(c[:, 2], -1.0, 1.0))
    e_a = np.stack([-np.sin(ra), np.cos(ra), np.zeros_like(ra)], axis=1)
    e_d = np.stack([-np.sin(dec) * np.cos(ra), -np.sin(dec) * np.sin(ra), np.cos(dec)], axis=1)
    return e_a, e_d


# --------------------------------------------------------------------------- catalogs
def randoms(n: int, footprint: Footprint = Footprint(), seed: int = 0) -> np.ndarray:
    """Uniform random catalog of ``n`` points within the footprint."""
    ra, dec = footprint.uniform(_rngs(seed)["randoms"], n)
    return radec_to_xyz(ra, dec)


def clustered(n: int, n_clusters: int, sigma_deg: float, footprint: Footprint = Footprint(),
              seed: int = 0, clustered_fraction: float = 0.7) -> np.ndarray:
    """Clustered data catalog.

    ``round(clustered_fraction * n)`` points are assigned uniformly at random to
    ``n_clusters`` centres (uniform in the footprint).  Each member is offset on
    the tangent plane at its centre by two independent N(0, sigma^2) draws along
    the RA and Dec directions and projected back to the sphere (gnomonic).
    Members that fall outside the footprint are redrawn.  The remaining points
    are uniform background in the footprint.
    """
    g = _rngs(seed)
    n_cl = int(round(clustered_fraction * n)) if n_clusters > 0 else 0
    cra, cdec = footprint.uniform(g["centres"], max(n_clusters, 1))
    centres = radec_to_xyz(cra, cdec)
    member_of = g["memberships"].integers(0, max(n_clusters, 1), n_cl)
    sig = sigma_deg * DEG
    ra = np.empty(n_cl)
    dec = np.empty(n_cl)
    todo = np.arange(n_cl)
    off = g["offsets"]
    for _ in range(1000):
        if todo.size == 0:
            break
        c = centres[member_of[todo]]
        e_a, e_d = _tangent_basis(c)
        xi = off.normal(0.0, sig, todo.size)
        eta = off.normal(0.0, sig, todo.size)
        v = c + xi[:, None] * e_a + eta[:, None] * e_d
        v /= np.linalg.norm(v, axis=1)[:, None]
        r, d = _xyz_to_radec(v)
        ok = footprint.contains(r, d)
        ra[todo[ok]] = r[ok]
        dec[todo[ok]] = d[ok]
        todo = todo[~ok]
    if todo.size:
        raise RuntimeError("cluster members could not be placed inside the footprint")
    bra, bdec = footprint.uniform(g["background"], n - n_cl)
    return radec_to_xyz(np.concatenate([ra, bra]), np.concatenate([dec, bdec]))


# --------------------------------------------------------------------------- bin edges
def linear_edges(theta_min_deg: float, theta_max_deg: float, nbins: int) -> np.ndarray:
    """``nbins + 1`` edges, linear in degrees, returned in radians (float64).

    t_k = (theta_min + k (theta_max - theta_min) / nbins) * pi/180, with both
    end points set to exactly theta_min*pi/180 and theta_max*pi/180.
    """
    k = np.arange(nbins + 1, dtype=np.float64)
    t = (theta_min_deg + k * ((theta_max_deg - theta_min_deg) / nbins)) * DEG
    t[0] = theta_min_deg * DEG
    t[-1] = theta_max_deg * DEG
    return t


def log_edges(theta_min_deg: float, theta_max_deg: float, nbins: int) -> np.ndarray:
    """``nbins + 1`` edges, logarithmic in degrees, returned in radians (float64)."""
    k = np.arange(nbins + 1, dtype=np.float64)
    step = math.log10(theta_max_deg / theta_min_deg) / nbins
    t = theta_min_deg * np.power(10.0, k * step) * DEG
    t[0] = theta_min_deg * DEG
    t[-1] = theta_max_deg * DEG
    return t


# --------------------------------------------------------------------------- named workloads
@dataclasses.dataclass
class Workload:
    name: str
    data: np.ndarray
    rand: np.ndarray
    edges: np.ndarray

    @property
    def pairs(self) -> int:
        nd, nr = len(self.data), len(self.rand)
        return nd * (nd - 1) // 2 + nr * (nr - 1) // 2 + nd * nr


def octant_small(seed: int = 0, n: int = 8192) -> Workload:
    """N_D = N_R = 8192 on the octant; 128 clusters, sigma 0.5 deg; 40 linear bins 0-10 deg."""
    fp = Footprint("octant")
    return Workload(f"octant_small_n{n}", clustered(n, 128, 0.5, fp, seed),
                    randoms(n, fp, seed), linear_edges(0.0, 10.0, 40))


def octant_precision(seed: int = 0, n: int = 1_000_000) -> Workload:
    """N_D = N_R = 1e6 on the octant; 1024 clusters, sigma 0.2 deg; 64 log bins 0.01-10 deg."""
    fp = Footprint("octant")
    return Workload(f"octant_precision_n{n}", clustered(n, 1024, 0.2, fp, seed),
                    randoms(n, fp, seed), log_edges(0.01, 10.0, 64))


def sphere_large(seed: int = 0, nd: int = 4_000_000, nr: int = 8_000_000) -> Workload:
    """Full sphere: 4e6 clustered data (4096 clusters, sigma 0.1 deg), 8e6 randoms; 80 log bins 0.005-2 deg."""
    fp = Footprint("sphere")
    return Workload(f"sphere_large_nd{nd}_nr{nr}", clustered(nd, 4096, 0.1, fp, seed),
                    randoms(nr, fp, seed), log_edges(0.005, 2.0, 80))


def jackknife_patches(seed: int = 0, nd: int = 2_000_000, npatch: int = 512,
                      lo: int = 1000, hi: int = 200_000, median: float = 2500.0,
                      s: float = 1.0) -> tuple[np.ndarray, np.ndarray, np.ndarray, np.ndarray]:
    """Octant catalog split into ``npatch`` sky patches of uneven occupancy.

    Patch data sizes are lognormal (``median``, shape ``s``), clipped to
    [lo, hi] and rescaled so they sum to ``nd`` exactly; each patch gets twice
    as many randoms.  Points are ordered by (Dec band, RA) and cut into
    contiguous chunks, so each patch is a compact sky region.

    Returns ``(data, rand, data_offsets, rand_offsets)`` where patch p holds
    ``data[data_offsets[p]:data_offsets[p+1]]`` and likewise for randoms.
    """
    g = _rngs(seed)
    sizes = np.clip(g["patches"].lognormal(math.log(median), s, npatch), lo, hi)
    sizes = _rescale_sizes(sizes, nd, lo, hi)
    fp = Footprint("octant")
    data = clustered(nd, 1024, 0.2, fp, seed)
    rand = randoms(2 * nd, fp, seed)
    data = _band_sort(data)
    rand = _band_sort(rand)
    doff = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    roff = 2 * doff
    return data, rand, doff, roff


def _rescale_sizes(sizes: np.ndarray, total: int, lo: int, hi: int) -> np.ndarray:
    s = sizes.astype(np.float64)
    for _ in range(100):
        s = np.clip(s * (total / s.sum()), lo, hi)
    out = np.floor(s).astype(np.int64)
    rem = total - int(out.sum())
    order = np.argsort(-(s - out))
    i = 0
    while rem != 0:
        k = order[i % len(order)]
        step = 1 if rem > 0 else -1
        if lo <= out[k] + step <= hi:
            out[k] += step
            rem -= step
        i += 1
    return out


def _band_sort(xyz: np.ndarray, nbands: int = 23) -> np.ndarray:
    ra, dec = _xyz_to_radec(xyz)
    band = np.minimum((dec / 90.0 * nbands).astype(np.int64), nbands - 1)
    order = np.lexsort((ra, band))
    return np.ascontiguousarray(xyz[order])


def serving_jobs(njobs: int = 2000, seed: int = 0, nd_min: float = 1e3, nd_max: float = 1e6,
                 rate_hz: float = 1.0) -> list[dict]:
    """Job descriptions for a Poisson-arrival pair-count stream.

    Each job has N_D log-uniform in [nd_min, nd_max], N_R = 2 N_D, a random cap
    footprint of radius U[5, 30] deg, 128 clusters with sigma 0.5 deg, and a
    per-job number of linear bins U{20..80} over 0-2 deg.  Catalogs are not
    materialised here; ``materialise_job`` builds one job's arrays.
    """
    g = _rngs(seed)["jobs"]
    t = np.cumsum(g.exponential(1.0 / rate_hz, njobs))
    nd = np.exp(g.uniform(math.log(nd_min), math.log(nd_max), njobs)).astype(np.int64)
    radius = g.uniform(5.0, 30.0, njobs)
    cra = g.uniform(0.0, 360.0, njobs)
    cdec = np.degrees(np.arcsin(g.uniform(-1.0, 1.0, njobs)))
    nb = g.integers(20, 81, njobs)
    return [dict(id=i, arrival_s=float(t[i]), nd=int(nd[i]), nr=int(2 * nd[i]),
                 footprint=Footprint("cap", float(cra[i]), float(cdec[i]), float(radius[i])),
                 nbins=int(nb[i]), seed=seed * 100003 + i) for i in range(njobs)]


def materialise_job(job: dict) -> Workload:
    fp = job["footprint"]
    d = clustered(job["nd"], 128, 0.5, fp, job["seed"])
    r = randoms(job["nr"], fp, job["seed"])
    return Workload(f"job{job['id']}", d, r, linear_edges(0.0, 2.0, job["nbins"]))


# --------------------------------------------------------------------------- 3-D variant
def box_points(n: int, side: float, seed: int = 0) -> np.ndarray:
    """Uniform points in the cube [0, side)^3 (3-D randoms)."""
    return _rngs(seed)["randoms"].uniform(0.0, side, (n, 3))


def box_clustered(n: int, n_clusters: int, sigma: float, side: float, seed: int = 0,
                  clustered_fraction: float = 0.7) -> np.ndarray:
    """Clustered 3-D points in the cube [0, side)^3: ``round(clustered_fraction * n)``
    members of ``n_clusters`` centres (uniform in the cube), offset by isotropic
    Gaussians of width ``sigma`` and redrawn when they leave the cube; the rest
    uniform."""
    g = _rngs(seed)
    n_cl = int(round(clustered_fraction * n)) if n_clusters > 0 else 0
    centres = g["centres"].uniform(0.0, side, (max(n_clusters, 1), 3))
    member_of = g["memberships"].integers(0, max(n_clusters, 1), n_cl)
    pts = np.empty((n_cl, 3))
    todo = np.arange(n_cl)
    for _ in range(1000):
        if todo.size == 0:
            break
        p = centres[member_of[todo]] + g["offsets"].normal(0.0, sigma, (todo.size, 3))
        ok = np.all((p >= 0.0) & (p < side), axis=1)
        pts[todo[ok]] = p[ok]
        todo = todo[~ok]
    if todo.size:
        raise RuntimeError("cluster members could not be placed inside the box")
    return np.concatenate([pts, g["background"].uniform(0.0, side, (n - n_cl, 3))])


def log_edges_r(r_min: float, r_max: float, nbins: int) -> np.ndarray:
    """Log-spaced distance edges with the endpoints exactly r_min and r_max."""
    t = r_min * 10.0 ** (np.arange(nbins + 1) * (math.log10(r_max / r_min) / nbins))
    t[0], t[-1] = r_min, r_max
    return t


def box_precision(seed: int = 0, n: int = 1_000_000, side: float = 1000.0) -> Workload:
    """3-D workload: n clustered points (4096 clusters of sigma 2) and n uniform
    points in a cube of side 1000, 30 log distance bins 0.5-50."""
    return Workload(f"box_n{n}", box_clustered(n, 4096, 2.0, side, seed), box_points(n, side, seed + 1),
                    log_edges_r(0.5, 50.0, 30))

