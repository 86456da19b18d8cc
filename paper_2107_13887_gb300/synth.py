"""Seeded synthetic meshes and displacements for the icing RBF deformation workloads.

This module only builds inputs: surface points, volume points, their wall
distances and prescribed surface displacements.  It holds none of the
method's arithmetic (no basis function, no greedy selection, no blending) so
that both the CUDA path and the CPU oracle can be fed from it.

Geometry follows the paper's test cases (Section 5): a NACA0012 airfoil of
chord 1 with points clustered at the leading and trailing edges, a structured
O-mesh around it, and a swept, tapered wing with NACA0012 sections.  The ice
shapes of the paper come from PoliMIce and are not available, so localised
Gaussian ice horns / ridges along the arc length from the leading edge stand
in for them.  The global benchmark motions are the sinusoids of Section 5.1
and Eq. 27, plus a rigid pitch and heave.

Wall distance ``d`` is the distance from a volume point to its nearest surface
vertex (a k-d tree query); the paper treats ``d(r)`` as given (Section 4).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "Case",
    "naca0012_surface",
    "airfoil_case",
    "wing_case",
    "make_config",
    "make_config_set",
    "CONFIGS",
    "CONFIG_SETS",
]


@dataclasses.dataclass
class Case:
    """One deformation problem: surface, displacement, volume and parameters."""

    name: str
    dim: int
    xyz_s: np.ndarray  # [n_s, dim] float64
    dS: np.ndarray  # [n_s, dim] float64
    xyz_v: np.ndarray  # [n_v, dim] float32
    d_v: np.ndarray  # [n_v] float32, wall distance
    R: list  # support radius per level
    eps: float
    D: float  # support distance cap of the wall-distance function (0 = none)
    k: float  # volume reduction factor (0 = use D at every level)
    nc_cap: int = 0  # most controls per level (0: the library's default)

    @property
    def n_s(self) -> int:
        return int(self.xyz_s.shape[0])

    @property
    def n_v(self) -> int:
        return int(self.xyz_v.shape[0])

    @property
    def n_levels(self) -> int:
        return len(self.R)


# ---------------------------------------------------------------- geometry


def _naca00_thickness(x: np.ndarray, t: float = 0.12) -> np.ndarray:
    """Half thickness of a symmetric NACA 4-digit section (open trailing edge)."""
    return 5.0 * t * (
        0.2969 * np.sqrt(x) - 0.1260 * x - 0.3516 * x**2 + 0.2843 * x**3 - 0.1015 * x**4
    )


def naca0012_surface(n: int):
    """Closed-loop NACA0012 outline of ``n`` points, chord 1, LE at the origin.

    Order: trailing edge (upper) -> leading edge -> trailing edge (lower), as
    in the usual Selig ordering; cosine clustering puts points near both the
    leading and the trailing edge.  No point is duplicated (the section has an
    open trailing edge), so no two surface points coincide.

    Returns (xy [n,2], outward unit normal [n,2], signed arc length from the
    leading edge [n]).
    """
    if n < 4:
        raise ValueError("need at least 4 surface points")
    n_up = n // 2
    n_lo = n - n_up
    # upper: x from 1 to ~0 (exclusive of the exact LE for one side)
    bu = np.linspace(0.0, math.pi, n_up, endpoint=False)  # beta in [0, pi)
    xu = 0.5 * (1.0 + np.cos(bu))  # 1 -> ~0
    bl = np.linspace(0.0, math.pi, n_lo + 1)[1:]  # (0, pi]
    xl = 0.5 * (1.0 - np.cos(bl))  # ~0 -> 1
    # place the exact leading edge (x = 0) on the lower sweep's first point
    xl = np.concatenate([[0.0], xl[:-1]]) if n_lo > 1 else np.array([0.0])
    yu = _naca00_thickness(xu)
    yl = -_naca00_thickness(xl)
    x = np.concatenate([xu, xl])
    y = np.concatenate([yu, yl])
    xy = np.stack([x, y], axis=1)
    # normals from central differences of the closed loop (counter-clockwise
    # ordering is upper TE->LE->lower TE, i.e. clockwise around the body, so the
    # outward normal is the tangent rotated by +90 degrees)
    t = np.roll(xy, -1, axis=0) - np.roll(xy, 1, axis=0)
    t[0] = xy[1] - xy[0]
    t[-1] = xy[-1] - xy[-2]
    nrm = np.stack([-t[:, 1], t[:, 0]], axis=1)
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    # make sure they point away from the chord line
    centre = np.array([0.5, 0.0])
    flip = np.einsum("ij,ij->i", nrm, xy - centre) < 0
    nrm[flip] *= -1.0
    # arc length, zero at the leading edge, negative on the upper side
    seg = np.linalg.norm(np.diff(xy, axis=0), axis=1)
    s = np.concatenate([[0.0], np.cumsum(seg)])
    i_le = int(np.argmin(x))
    s = s - s[i_le]
    return xy, nrm, s


def _geometric_heights(n_layers: int, h1: float, H: float) -> np.ndarray:
    """Wall-normal heights h_1..h_n growing geometrically from h1 to H."""
    lo, hi = 1.0 + 1e-12, 4.0
    for _ in range(200):  # bisection on the growth ratio
        q = 0.5 * (lo + hi)
        e = n_layers * math.log(q)
        tot = h1 * math.expm1(e) / (q - 1.0) if e < 700.0 else math.inf
        if tot > H:
            hi = q
        else:
            lo = q
    q = 0.5 * (lo + hi)
    return h1 * (q ** np.arange(1, n_layers + 1) - 1.0) / (q - 1.0)


def _wall_distance(xyz_v: np.ndarray, xyz_s: np.ndarray) -> np.ndarray:
    from scipy.spatial import cKDTree

    tree = cKDTree(xyz_s)
    d, _ = tree.query(xyz_v, k=1, workers=-1)
    return d


def _o_mesh(xy, nrm, n_layers, radius, h1=1e-5, reach=0.5):
    """Structured O-mesh: each surface point marched out in ``n_layers`` layers.

    Near the wall the layers follow the surface normal; further out they blend
    (smoothstep over the first ``reach`` of the radius) into rays to a
    far-field circle of ``radius`` about mid-chord, on which the surface
    points are spread evenly by arc length, so neighbouring rays never meet
    (the blunt trailing edge included).  Layout [surface point][layer].
    """
    h = _geometric_heights(n_layers, h1, radius)
    centre = np.array([0.5, 0.0])
    seg = np.linalg.norm(np.roll(xy, -1, axis=0) - xy, axis=1)
    s = np.concatenate([[0.0], np.cumsum(seg)[:-1]])
    ang = 2.0 * math.pi * s / seg.sum() + math.atan2(xy[0, 1] - centre[1], xy[0, 0] - centre[0])
    far = centre + radius * np.stack([np.cos(ang), np.sin(ang)], axis=1)
    w = (h / radius)[None, :, None]  # 0 at wall .. 1 at far field
    near = xy[:, None, :] + nrm[:, None, :] * h[None, :, None]
    ray = xy[:, None, :] + (far - xy)[:, None, :] * w
    x = np.clip(w / reach, 0.0, 1.0)
    blend = x * x * (3.0 - 2.0 * x)
    pts = (1.0 - blend) * near + blend * ray
    return pts.reshape(-1, 2)


# ----------------------------------------------------------- displacements


def _ice_bumps(s, nrm, rng, peaks, centres, sigma, jitter=0.1):
    """Sum of Gaussian horns in arc length along the outward normal.

    Each horn's peak and width are scaled by U[1-jitter, 1+jitter] and its
    centre is shifted by U[-jitter, jitter] widths, all drawn from ``rng``: the
    shape stays smooth, and the shift breaks the upper/lower symmetry of the
    section so that no two surface errors tie exactly.
    """
    amp = np.zeros_like(s)
    for p, c in zip(peaks, centres):
        pj = p * rng.uniform(1.0 - jitter, 1.0 + jitter)
        sj = sigma * rng.uniform(1.0 - jitter, 1.0 + jitter)
        cj = c + sigma * rng.uniform(-jitter, jitter)
        amp += pj * np.exp(-0.5 * ((s - cj) / sj) ** 2)
    return nrm * amp[:, None]


def airfoil_case(
    n_surf: int,
    n_layers: int,
    displacement: str = "bump",
    seed: int = 0,
    R=(0.5,),
    eps: float = 1e-4,
    D: float = 2.0,
    k: float = 0.0,
    radius: float = 20.0,
    name: str | None = None,
    wall_distance: bool = True,
) -> Case:
    """2D NACA0012 airfoil in an O-mesh with a prescribed surface displacement.

    displacement:
      ``bump``         one Gaussian ice horn at the leading edge, peak 0.02,
                        sigma 0.03 along the arc length, normal direction,
                        peak, width and centre jittered by 10% from the seed;
      ``horns``        three Gaussian horns, peaks U[0.01, 0.04], centres
                        U[-0.06, 0.06] in arc length, sigma 0.03, same jitter;
      ``pitch_heave``  rigid pitch of 5 degrees about the quarter chord plus
                        a heave of 0.05 chord;
      ``sinusoid``     dy = 0.01 sin(15 pi x) (the 2D benchmark of Section 5.1).
    """
    rng = np.random.default_rng(seed)
    xy, nrm, s = naca0012_surface(n_surf)
    if displacement == "bump":
        dS = _ice_bumps(s, nrm, rng, [0.02], [0.0], 0.03)
    elif displacement == "horns":
        peaks = rng.uniform(0.01, 0.04, size=3)
        centres = rng.uniform(-0.06, 0.06, size=3)
        dS = _ice_bumps(s, nrm, rng, peaks, centres, 0.03)
    elif displacement == "pitch_heave":
        a = math.radians(5.0)
        c, sn = math.cos(a), math.sin(a)
        q = np.array([0.25, 0.0])
        rel = xy - q
        rot = np.stack([c * rel[:, 0] + sn * rel[:, 1], -sn * rel[:, 0] + c * rel[:, 1]], axis=1)
        dS = rot - rel
        dS[:, 1] += 0.05
    elif displacement == "sinusoid":
        dS = np.zeros_like(xy)
        dS[:, 1] = 0.01 * np.sin(15.0 * math.pi * xy[:, 0])
    else:
        raise ValueError(displacement)
    if n_layers > 0:
        xv = _o_mesh(xy, nrm, n_layers, radius)
        d = _wall_distance(xv, xy) if wall_distance else None
    else:
        xv = np.zeros((0, 2))
        d = np.zeros((0,))
    return Case(
        name=name or f"naca0012_{n_surf}s_{xv.shape[0]}v_{displacement}",
        dim=2,
        xyz_s=np.ascontiguousarray(xy, dtype=np.float64),
        dS=np.ascontiguousarray(dS, dtype=np.float64),
        xyz_v=np.ascontiguousarray(xv, dtype=np.float32),
        d_v=None if d is None else np.ascontiguousarray(d, dtype=np.float32),
        R=list(R),
        eps=float(eps),
        D=float(D),
        k=float(k),
    )


def _wing_surface(n_chord, n_span, semi_span=3.0, sweep_deg=30.0, taper=0.5):
    xy, nrm2, s2 = naca0012_surface(n_chord)
    # spanwise stations clustered slightly toward root and tip
    u = 0.5 * (1.0 - np.cos(np.linspace(0.0, math.pi, n_span)))
    z = semi_span * u
    chord = 1.0 - (1.0 - taper) * (z / semi_span)
    xle = z * math.tan(math.radians(sweep_deg))
    X = xle[:, None] + chord[:, None] * xy[None, :, 0]
    Y = chord[:, None] * xy[None, :, 1]
    Z = np.broadcast_to(z[:, None], X.shape)
    pts = np.stack([X, Y, Z], axis=-1).reshape(-1, 3)
    nrm = np.concatenate([nrm2, np.zeros((n_chord, 1))], axis=1)
    nrm = np.broadcast_to(nrm[None], (n_span, n_chord, 3)).reshape(-1, 3)
    s = (chord[:, None] * s2[None, :]).reshape(-1)
    zz = Z.reshape(-1)
    return pts, np.ascontiguousarray(nrm), s, zz


def wing_case(
    n_chord: int,
    n_span: int,
    n_layers: int,
    displacement: str = "ridge",
    seed: int = 0,
    R=(1.5, 0.4, 0.1),
    eps: float = 1e-5,
    D: float = 1.0,
    k: float = 4.0,
    radius: float = 20.0,
    semi_span: float = 3.0,
    name: str | None = None,
    wall_distance: bool = True,
    nc_cap: int = 0,
) -> Case:
    """3D swept (30 deg), tapered (0.5) wing of NACA0012 sections, span 3 chords.

    The volume is an O-H grid standing in for the paper's unstructured C-H
    mesh: at every span station the section's points carry ``n_layers``
    geometric layers (first height 1e-5, last ``radius``) that follow the
    normals near the wall and blend into rays to a far-field circle, the
    layers of the unit-chord section's O-mesh.  Layout [span][chord][layer].

    displacement:
      ``ridge``     leading-edge ice ridge, height growing linearly from 0.01
                    at the root to 0.03 at the tip with seeded smooth spanwise
                    noise (three sine modes, +-15% in total), chordwise
                    Gaussian of sigma 0.02 in arc length, its centre shifted
                    by a seeded U[-0.1, 0.1] sigma off the leading edge;
      ``sinusoid``  dy = 0.03 sin(4 pi z) (Eq. 27).
    """
    rng = np.random.default_rng(seed)
    pts, nrm, s, z = _wing_surface(n_chord, n_span, semi_span=semi_span)
    if displacement == "ridge":
        w = rng.uniform(-1.0, 1.0, size=3)
        ph = rng.uniform(0.0, 2.0 * math.pi, size=3)
        noise = 1.0 + 0.05 * sum(
            w[m] * np.sin((m + 1) * math.pi * z / semi_span + ph[m]) for m in range(3)
        )
        h = (0.01 + 0.02 * z / semi_span) * noise
        # the ridge's centre shifted by a seeded tenth of its width at most:
        # the upper and lower sides then never carry exactly equal errors
        s0 = 0.02 * rng.uniform(-0.1, 0.1)
        amp = h * np.exp(-0.5 * ((s - s0) / 0.02) ** 2)
        dS = nrm * amp[:, None]
    elif displacement == "sinusoid":
        dS = np.zeros_like(pts)
        dS[:, 1] = 0.03 * np.sin(4.0 * math.pi * z)
    else:
        raise ValueError(displacement)
    if n_layers > 0:
        # every span station carries the layers of the unit-chord section's
        # O-mesh, as offsets from its surface points
        xy2, nrm2, _ = naca0012_surface(n_chord)
        off = _o_mesh(xy2, nrm2, n_layers, radius).reshape(n_chord, n_layers, 2) - xy2[:, None, :]
        off3 = np.concatenate([off, np.zeros((n_chord, n_layers, 1))], axis=2)
        xv = (pts.reshape(n_span, n_chord, 1, 3) + off3[None]).reshape(-1, 3)
        d = _wall_distance(xv, pts) if wall_distance else None
    else:
        xv = np.zeros((0, 3))
        d = np.zeros((0,))
    return Case(
        name=name or f"wing_{pts.shape[0]}s_{xv.shape[0]}v_{displacement}",
        dim=3,
        xyz_s=np.ascontiguousarray(pts, dtype=np.float64),
        dS=np.ascontiguousarray(dS, dtype=np.float64),
        xyz_v=np.ascontiguousarray(xv, dtype=np.float32),
        d_v=None if d is None else np.ascontiguousarray(d, dtype=np.float32),
        R=list(R),
        eps=float(eps),
        D=float(D),
        k=float(k),
        nc_cap=int(nc_cap),
    )


# ------------------------------------------------------------- named configs

CONFIGS = {
    # 2D plain FP64: 400 surface points, 400x100 O-mesh to radius 20, one ice horn
    "naca0012_400s_40kv_bump": dict(
        kind="airfoil", n_surf=400, n_layers=100, displacement="bump", R=(0.5,), eps=1e-4, D=2.0, k=0.0
    ),
    # 2D global vs local: 4000 surface points, 4000x250 = 1M volume points, two levels
    "naca0012_4000s_1mv_pitch_heave": dict(
        kind="airfoil", n_surf=4000, n_layers=250, displacement="pitch_heave", R=(1.0, 0.2), eps=1e-5, D=2.0, k=5.0
    ),
    "naca0012_4000s_1mv_horns": dict(
        kind="airfoil", n_surf=4000, n_layers=250, displacement="horns", R=(1.0, 0.2), eps=1e-5, D=2.0, k=5.0
    ),
    # 3D swept wing: 400x150 = 60k surface points, 60k x 100 = 6M volume points, three levels
    "wing_60ks_6mv_ridge": dict(
        kind="wing", n_chord=400, n_span=150, n_layers=100, displacement="ridge", R=(1.5, 0.4, 0.1), eps=1e-5, D=1.0, k=4.0
    ),
}


# Workloads of several meshes deformed together
CONFIG_SETS = {
    # four swept wings of uneven size, seeds 0-3: 200x150 = 30k, 400x200 =
    # 80k, 500x300 = 150k and 625x400 = 250k surface points, 100 layers each
    # (3M, 8M, 15M, 25M volume points, float32), the ridge of the 60k wing,
    # three levels, at most 20,000 controls per level
    "wings4_30k_250ks_3m_25mv_ridge": [
        dict(kind="wing", n_chord=nc, n_span=ns, n_layers=100, displacement="ridge", R=(1.5, 0.4, 0.1), eps=1e-5,
             D=1.0, k=4.0, nc_cap=20000, seed=s)
        for s, (nc, ns) in enumerate([(200, 150), (400, 200), (500, 300), (625, 400)])
    ],
}


def make_config_set(name: str, n_layers: int | None = None, wall_distance: bool = True, **over):
    """Build a named workload of several meshes (a list of Case).  With
    wall_distance = False the volumes carry no wall distances (d_v = None):
    the library computes them on the device."""
    out = []
    for i, spec in enumerate(CONFIG_SETS[name]):
        spec = dict(spec)
        spec.update(over)
        if n_layers is not None:
            spec["n_layers"] = n_layers
        spec.pop("kind")
        out.append(wing_case(name=f"{name}[{i}]", wall_distance=wall_distance, **spec))
    return out


def make_config(name: str, seed: int = 0, n_layers: int | None = None, **over) -> Case:
    """Build a named workload.  ``n_layers`` (or other keys) may be overridden
    to make reduced-size variants of the same shape for tests."""
    spec = dict(CONFIGS[name])
    spec.update(over)
    if n_layers is not None:
        spec["n_layers"] = n_layers
    kind = spec.pop("kind")
    if kind == "airfoil":
        return airfoil_case(seed=seed, name=name, **spec)
    return wing_case(seed=seed, name=name, **spec)
