"""Seeded synthetic inputs for the nonoverlapping DDM-ELM solver.

This module produces the *inputs* of the method and nothing else: the
subdomain decomposition of the unit square, the collocation points of every
subdomain (interior, outer-boundary and interface points, Section 3), the
outward interface normals, the map from each local interface row to its
global interface unknown u_Gamma, the randomly drawn hidden-layer parameters
theta^s = (w^s_j, b^s_j) (the "Set theta^s randomly" step of Algorithm 1,
with the initialisation of Eq. (4.3)), the source/boundary data f, g at the
points, and the test points with their exact solution.

It contains none of the method's arithmetic (no features, no least squares,
no Schur complement) and imports neither the CUDA binding nor the oracle;
both of those consume what it returns.

Layout conventions shared by every consumer:

* Subdomain s = iy * gx + ix covers [ix/gx, (ix+1)/gx] x [iy/gy, (iy+1)/gy].
* Rows of subdomain s are ordered [interior | boundary | interface], matching
  the row blocks of K^s in Section 3; ``counts[s] = (m_i, m_b, m_Gamma)``.
  Arrays are padded to ``m_max`` rows; padded rows have zero coordinates,
  zero normals and dof = -1.
* Points on an edge sit at cell centres (k + 1/2)/p along the edge, so no
  collocation point is a corner or cross point.
* Interface edges are numbered globally: vertical edges (between (ix,iy) and
  (ix+1,iy)) first, id = iy*(gx-1) + ix, then horizontal edges (between
  (ix,iy) and (ix,iy+1)), id = (gx-1)*gy + iy*gx + ix.  The k-th point of
  edge e is global interface unknown e*p_ifc + k.  Both subdomains sharing
  an edge produce bit-identical coordinates for that point.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

# Edge order inside a subdomain: left, right, bottom, top.
_EDGES = ("left", "right", "bottom", "top")
_NORMALS = {"left": (-1.0, 0.0), "right": (1.0, 0.0),
            "bottom": (0.0, -1.0), "top": (0.0, 1.0)}


@dataclasses.dataclass
class FluxRows:
    """Explicit rows of the A^s blocks (the normal-derivative rows of Section 3), for
    decompositions with cross points (the remark in Section 3: at a point where several
    edges meet, A^s gets one row per edge through it, with that edge's normal).  Row f of
    subdomain s sits at its interface row ``row[s, f]`` (an index among the interface
    rows) with normal ``nrm[s, f]``; ``fdof[s, f]`` is the global flux condition it
    belongs to, and every condition sums the rows of the two subdomains of its edge.
    Without it, each interface row carries one row with its own normal and the condition
    of its interface unknown."""
    n_flux: int
    count: np.ndarray       # int32 [N]
    row: np.ndarray         # int32 [N, f_max]
    nrm: np.ndarray         # float64 [N, f_max, 2]
    fdof: np.ndarray        # int32 [N, f_max], -1 past count


@dataclasses.dataclass
class Geometry:
    """Decomposition of the unit square and the collocation points."""
    gx: int
    gy: int
    mi_x: int
    mi_y: int
    p_bnd: int
    p_ifc: int
    counts: np.ndarray      # int32 [N, 3] = (m_i, m_b, m_Gamma)
    xy: np.ndarray          # float64 [N, m_max, 2]
    nrm: np.ndarray         # float64 [N, m_max, 2], outward normal on interface rows
    dof: np.ndarray         # int32 [N, m_max], global interface unknown or -1
    n_gamma: int
    flux: Optional[FluxRows] = None   # explicit A^s rows (cross points), else one per interface row

    @property
    def n_sub(self) -> int:
        return self.gx * self.gy

    @property
    def m_max(self) -> int:
        return int(self.xy.shape[1])

    def rows(self, s: int):
        """(interior, boundary, interface) row slices of subdomain s."""
        mi, mb, mg = (int(v) for v in self.counts[s])
        return slice(0, mi), slice(mi, mi + mb), slice(mi + mb, mi + mb + mg)

    def box(self, s: int):
        ix, iy = s % self.gx, s // self.gx
        return (ix / self.gx, (ix + 1) / self.gx, iy / self.gy, (iy + 1) / self.gy)


def _edge_points(gx, gy, ix, iy, edge, p):
    """Cell-centred points along one edge of subdomain (ix, iy)."""
    t = (np.arange(p, dtype=np.float64) + 0.5) / p
    if edge in ("left", "right"):
        xe = (ix + (1 if edge == "right" else 0)) / gx
        return np.stack([np.full(p, xe), (iy + t) / gy], axis=1)
    ye = (iy + (1 if edge == "top" else 0)) / gy
    return np.stack([(ix + t) / gx, np.full(p, ye)], axis=1)


def _edge_id(gx, gy, ix, iy, edge):
    """Global id of the interface edge, or None if the edge is on the outer boundary."""
    if edge == "left":
        return None if ix == 0 else iy * (gx - 1) + (ix - 1)
    if edge == "right":
        return None if ix == gx - 1 else iy * (gx - 1) + ix
    if edge == "bottom":
        return None if iy == 0 else (gx - 1) * gy + (iy - 1) * gx + ix
    return None if iy == gy - 1 else (gx - 1) * gy + iy * gx + ix


def make_geometry(gx: int, gy: int, mi_x: int, mi_y: int, p_bnd: int, p_ifc: int,
                  m_max: Optional[int] = None) -> Geometry:
    """Build the point sets of a gx x gy decomposition of (0,1)^2."""
    n = gx * gy
    per = []
    for s in range(n):
        ix, iy = s % gx, s // gx
        tx = (np.arange(mi_x, dtype=np.float64) + 0.5) / mi_x
        ty = (np.arange(mi_y, dtype=np.float64) + 0.5) / mi_y
        X, Y = np.meshgrid((ix + tx) / gx, (iy + ty) / gy, indexing="xy")
        interior = np.stack([X.ravel(), Y.ravel()], axis=1)
        bnd, ifc, nrm, dof = [], [], [], []
        for e in _EDGES:
            eid = _edge_id(gx, gy, ix, iy, e)
            if eid is None:
                if p_bnd > 0:
                    bnd.append(_edge_points(gx, gy, ix, iy, e, p_bnd))
            else:
                ifc.append(_edge_points(gx, gy, ix, iy, e, p_ifc))
                nrm.append(np.tile(np.array(_NORMALS[e]), (p_ifc, 1)))
                dof.append(eid * p_ifc + np.arange(p_ifc))
        bnd = np.concatenate(bnd) if bnd else np.zeros((0, 2))
        ifc = np.concatenate(ifc) if ifc else np.zeros((0, 2))
        nrm = np.concatenate(nrm) if nrm else np.zeros((0, 2))
        dof = np.concatenate(dof).astype(np.int32) if dof else np.zeros(0, np.int32)
        per.append((interior, bnd, ifc, nrm, dof))
    need = max(len(a) + len(b) + len(c) for a, b, c, _, _ in per)
    m_max = need if m_max is None else m_max
    if m_max < need:
        raise ValueError(f"m_max={m_max} < rows needed {need}")
    counts = np.zeros((n, 3), np.int32)
    xy = np.zeros((n, m_max, 2))
    nr = np.zeros((n, m_max, 2))
    dd = np.full((n, m_max), -1, np.int32)
    for s, (interior, bnd, ifc, nrm, dof) in enumerate(per):
        mi, mb, mg = len(interior), len(bnd), len(ifc)
        counts[s] = (mi, mb, mg)
        xy[s, :mi] = interior
        xy[s, mi:mi + mb] = bnd
        xy[s, mi + mb:mi + mb + mg] = ifc
        nr[s, mi + mb:mi + mb + mg] = nrm
        dd[s, mi + mb:mi + mb + mg] = dof
    n_gamma = ((gx - 1) * gy + gx * (gy - 1)) * p_ifc
    return Geometry(gx, gy, mi_x, mi_y, p_bnd, p_ifc, counts, xy, nr, dd, n_gamma)


# --------------------------------------------------------------------------
# Hidden-layer parameters theta^s (Algorithm 1, first step; Eq. (4.3))
# --------------------------------------------------------------------------

def draw_theta(geom: Geometry, n_neurons: int, mode: str, seed: int,
               c: float = 1.0 / 8.0, r_scale: float = 0.5):
    """Draw (W [N, n, 2], b [N, n]) in global coordinates.

    Modes
    -----
    ``paper``      Eq. (4.3): w ~ U([-l, l]^2) with l = c*sqrt(n), n = N*n_N the
                   total neuron count; b = -w . xi with xi uniform on the closed
                   r-neighbourhood of the subdomain, r = r_scale * diam(Omega_s)
                   (the paper uses r = diam/2).  xi is drawn by rejection from
                   the box enlarged by r.
    ``local_unit`` w_hat, b_hat ~ U(-1, 1) for the local coordinates
                   x_hat = 2 (x - centre) / h in [-1, 1]^2, then mapped to global
                   coordinates (w = 2 w_hat / h, b = b_hat - w . centre).
    ``global_unit`` w ~ U([-1, 1]^2), b ~ U(-1, 1) in global coordinates.
    ``he``         w ~ U([-l, l]^2) with l = sqrt(2 / n_N), b = 0 (Table 1 baseline).
    ``radial``     Remark 4.2: density proportional to |w| on
                   [-l, l]^2 (rejection sampling), b as in ``paper``.
    """
    rng = np.random.default_rng(seed)
    N = geom.n_sub
    W = np.zeros((N, n_neurons, 2))
    B = np.zeros((N, n_neurons))
    for s in range(N):
        x0, x1, y0, y1 = geom.box(s)
        hx, hy = x1 - x0, y1 - y0
        cx, cy = 0.5 * (x0 + x1), 0.5 * (y0 + y1)
        if mode == "local_unit":
            wh = rng.uniform(-1.0, 1.0, size=(n_neurons, 2))
            bh = rng.uniform(-1.0, 1.0, size=n_neurons)
            w = np.stack([2.0 * wh[:, 0] / hx, 2.0 * wh[:, 1] / hy], axis=1)
            W[s] = w
            B[s] = bh - (w[:, 0] * cx + w[:, 1] * cy)
        elif mode == "global_unit":
            W[s] = rng.uniform(-1.0, 1.0, size=(n_neurons, 2))
            B[s] = rng.uniform(-1.0, 1.0, size=n_neurons)
        elif mode == "he":
            lim = math.sqrt(2.0 / n_neurons)
            W[s] = rng.uniform(-lim, lim, size=(n_neurons, 2))
            B[s] = 0.0
        elif mode in ("paper", "radial"):
            lim = c * math.sqrt(N * n_neurons)
            if mode == "paper":
                w = rng.uniform(-lim, lim, size=(n_neurons, 2))
            else:
                w = np.zeros((n_neurons, 2))
                k = 0
                while k < n_neurons:
                    cand = rng.uniform(-lim, lim, size=(2 * n_neurons, 2))
                    acc = rng.uniform(0.0, 1.0, size=2 * n_neurons) * lim * math.sqrt(2.0)
                    cand = cand[np.hypot(cand[:, 0], cand[:, 1]) >= acc]
                    take = min(len(cand), n_neurons - k)
                    w[k:k + take] = cand[:take]
                    k += take
            r = r_scale * math.hypot(hx, hy)
            xi = np.zeros((n_neurons, 2))
            k = 0
            while k < n_neurons:
                cand = np.stack([rng.uniform(x0 - r, x1 + r, 2 * n_neurons),
                                 rng.uniform(y0 - r, y1 + r, 2 * n_neurons)], axis=1)
                dx = np.maximum(np.maximum(x0 - cand[:, 0], cand[:, 0] - x1), 0.0)
                dy = np.maximum(np.maximum(y0 - cand[:, 1], cand[:, 1] - y1), 0.0)
                cand = cand[dx * dx + dy * dy <= r * r]
                take = min(len(cand), n_neurons - k)
                xi[k:k + take] = cand[:take]
                k += take
            W[s] = w
            B[s] = -(w[:, 0] * xi[:, 0] + w[:, 1] * xi[:, 1])
        else:
            raise ValueError(f"unknown theta mode {mode!r}")
    return W, B


# --------------------------------------------------------------------------
# Right-hand sides: -Laplace(u) = f in (0,1)^2, u = g on the boundary
# --------------------------------------------------------------------------

@dataclasses.dataclass
class Source:
    """Manufactured or random source term with (when known) its exact solution."""
    kind: str
    params: dict

    def f(self, xy):
        coef = self.params.get("coef")
        if coef is not None and self.kind != "const":
            # -div(rho grad u) = -rho Lap u - grad rho . grad u for the closed-form u
            return (-coef.rho(xy) * self.lap_u(xy)
                    - (coef.grad(xy) * self.grad_u(xy)).sum(-1))
        x, y = xy[..., 0], xy[..., 1]
        if self.kind == "const":
            return np.full(x.shape, float(self.params.get("value", 1.0)))
        if self.kind == "sinsin":
            return 2.0 * math.pi ** 2 * np.sin(math.pi * x) * np.sin(math.pi * y)
        if self.kind == "sin2pi_exp":
            return (4.0 * math.pi ** 2 - 1.0) * np.sin(2.0 * math.pi * x) * np.exp(y)
        if self.kind == "fourier":
            a = self.params["a"]
            out = np.zeros_like(x)
            for k in range(a.shape[0]):
                for l in range(a.shape[1]):
                    out += a[k, l] * np.sin((k + 1) * math.pi * x) * np.sin((l + 1) * math.pi * y)
            return out
        if self.kind == "grf":
            a, w, b = self.params["a"], self.params["w"], self.params["b"]
            z = x[..., None] * w[:, 0] + y[..., None] * w[:, 1] + b
            return (a * np.sin(z)).sum(-1)
        raise ValueError(self.kind)

    def u(self, xy):
        x, y = xy[..., 0], xy[..., 1]
        if self.kind == "sinsin":
            return np.sin(math.pi * x) * np.sin(math.pi * y)
        if self.kind == "sin2pi_exp":
            return np.sin(2.0 * math.pi * x) * np.exp(y)
        if self.kind == "fourier":
            a = self.params["a"]
            out = np.zeros_like(x)
            for k in range(a.shape[0]):
                for l in range(a.shape[1]):
                    lam = math.pi ** 2 * ((k + 1) ** 2 + (l + 1) ** 2)
                    out += a[k, l] / lam * np.sin((k + 1) * math.pi * x) * np.sin((l + 1) * math.pi * y)
            return out
        raise ValueError(f"no closed-form solution for {self.kind}")

    def grad_u(self, xy):
        x, y = xy[..., 0], xy[..., 1]
        pi = math.pi
        if self.kind == "sinsin":
            return np.stack([pi * np.cos(pi * x) * np.sin(pi * y),
                             pi * np.sin(pi * x) * np.cos(pi * y)], axis=-1)
        if self.kind == "sin2pi_exp":
            return np.stack([2 * pi * np.cos(2 * pi * x) * np.exp(y),
                             np.sin(2 * pi * x) * np.exp(y)], axis=-1)
        if self.kind == "fourier":
            a = self.params["a"]
            gx_ = np.zeros_like(x)
            gy_ = np.zeros_like(x)
            for k in range(a.shape[0]):
                for l in range(a.shape[1]):
                    kk, ll = (k + 1) * pi, (l + 1) * pi
                    lam = kk * kk + ll * ll
                    gx_ += a[k, l] / lam * kk * np.cos(kk * x) * np.sin(ll * y)
                    gy_ += a[k, l] / lam * ll * np.sin(kk * x) * np.cos(ll * y)
            return np.stack([gx_, gy_], axis=-1)
        raise ValueError(f"no closed-form solution for {self.kind}")

    def lap_u(self, xy):
        """Laplacian of the closed-form solution."""
        x, y = xy[..., 0], xy[..., 1]
        pi = math.pi
        if self.kind == "sinsin":
            return -2.0 * pi ** 2 * np.sin(pi * x) * np.sin(pi * y)
        if self.kind == "sin2pi_exp":
            return (1.0 - 4.0 * pi ** 2) * np.sin(2.0 * pi * x) * np.exp(y)
        if self.kind == "fourier":
            a = self.params["a"]
            out = np.zeros_like(x)
            for k in range(a.shape[0]):
                for l in range(a.shape[1]):
                    out -= a[k, l] * np.sin((k + 1) * pi * x) * np.sin((l + 1) * pi * y)
            return out
        raise ValueError(f"no closed-form solution for {self.kind}")

    def g(self, xy):
        if self.kind in ("fourier", "grf", "const"):
            return np.zeros(xy.shape[:-1])
        return self.u(xy)

    @property
    def has_exact(self) -> bool:
        return self.kind in ("sinsin", "sin2pi_exp", "fourier")


# --------------------------------------------------------------------------
# Variable coefficient of -div(rho grad u) = f (Section 4, variable-coefficient
# Poisson): rho and grad rho at points; these are problem data, not the method
# --------------------------------------------------------------------------

@dataclasses.dataclass
class Coefficient:
    """``sine``: rho = 1 + amp sin(2 pi k . x) with an integer wave vector k.
    ``grf``: rho = tanh(grf(x)) + 1.1 with grf the approximate Gaussian random field of
    Eq. (4.5) (the paper's coefficient, between 0.1 and 2.1).
    ``const``: rho = value (reduces the operator to value * (-Laplacian))."""
    kind: str
    params: dict

    def _grf(self, xy):
        a, w, b = self.params["a"], self.params["w"], self.params["b"]
        z = xy[..., 0, None] * w[:, 0] + xy[..., 1, None] * w[:, 1] + b
        return (a * np.sin(z)).sum(-1), np.stack([(a * np.cos(z) * w[:, 0]).sum(-1),
                                                  (a * np.cos(z) * w[:, 1]).sum(-1)], axis=-1)

    def rho(self, xy):
        if self.kind == "sine":
            k, amp = self.params["k"], self.params["amp"]
            return 1.0 + amp * np.sin(2.0 * math.pi * (xy[..., 0] * k[0] + xy[..., 1] * k[1]))
        if self.kind == "grf":
            return np.tanh(self._grf(xy)[0]) + 1.1
        if self.kind == "const":
            return np.full(xy.shape[:-1], float(self.params["value"]))
        raise ValueError(self.kind)

    def grad(self, xy):
        if self.kind == "sine":
            k, amp = self.params["k"], self.params["amp"]
            c = amp * 2.0 * math.pi * np.cos(2.0 * math.pi * (xy[..., 0] * k[0] + xy[..., 1] * k[1]))
            return np.stack([c * k[0], c * k[1]], axis=-1)
        if self.kind == "grf":
            g, dg = self._grf(xy)
            return (1.0 - np.tanh(g) ** 2)[..., None] * dg
        if self.kind == "const":
            return np.zeros(xy.shape[:-1] + (2,))
        raise ValueError(self.kind)


def make_coefficient(kind: str, seed: int = 0, amp: float = 0.5, alpha: float = 16.0,
                     value: float = 1.0) -> Coefficient:
    """``sine``: k = (k1, k2) with k_i uniform in {1..4} (seeded); ``grf``: Eq. (4.5) with
    256 terms as make_source('grf'); ``const``: rho = value."""
    rng = np.random.default_rng(seed)
    if kind == "sine":
        return Coefficient(kind, {"k": rng.integers(1, 5, size=2).astype(np.float64), "amp": amp})
    if kind == "grf":
        a = rng.normal(0.0, alpha ** 2 / 16.0, size=256)
        w = rng.normal(0.0, alpha, size=(256, 2))
        b = rng.uniform(0.0, 2.0 * math.pi, size=256)
        return Coefficient(kind, {"a": a, "w": w, "b": b})
    if kind == "const":
        return Coefficient(kind, {"value": value})
    raise ValueError(kind)


def coef_rows(geom: Geometry, coef: Coefficient) -> np.ndarray:
    """Per-row coefficient data [N, m_max, 3] = (rho, d rho/dx, d rho/dy) at every
    collocation point (only interior rows enter the operator); zero on padding."""
    out = np.zeros((geom.n_sub, geom.m_max, 3))
    for s in range(geom.n_sub):
        m = int(geom.counts[s].sum())
        out[s, :m, 0] = coef.rho(geom.xy[s, :m])
        out[s, :m, 1:] = coef.grad(geom.xy[s, :m])
    return out


def make_source(kind: str, seed: int = 0, modes: int = 4, alpha: float = 16.0) -> Source:
    """``fourier``: f = sum_{k,l<=modes} a_kl sin(k pi x) sin(l pi y), a_kl ~ N(0,1),
    exact u = sum a_kl sin sin / (pi^2 (k^2+l^2)), g = 0.
    ``grf``: Eq. (4.5) with 256 terms, a_i ~ N(0, alpha^4/256), w_i ~ N(0, alpha^2 I),
    b_i ~ U(0, 2 pi), g = 0 (no closed form)."""
    rng = np.random.default_rng(seed)
    if kind == "fourier":
        return Source(kind, {"a": rng.standard_normal((modes, modes))})
    if kind == "grf":
        a = rng.normal(0.0, alpha ** 2 / 16.0, size=256)
        w = rng.normal(0.0, alpha, size=(256, 2))
        b = rng.uniform(0.0, 2.0 * math.pi, size=256)
        return Source(kind, {"a": a, "w": w, "b": b})
    if kind == "const":
        return Source(kind, {"value": 1.0})
    return Source(kind, {})


def rhs_rows(geom: Geometry, src: Source) -> np.ndarray:
    """Per-row data [N, m_max]: f at interior rows, g at boundary rows, 0 on
    interface rows and padding (the F^s of Section 3)."""
    out = np.zeros((geom.n_sub, geom.m_max))
    for s in range(geom.n_sub):
        ri, rb, _ = geom.rows(s)
        out[s, ri] = src.f(geom.xy[s, ri])
        out[s, rb] = src.g(geom.xy[s, rb])
    return out


def fourier_basis_rows(geom: Geometry, modes: int) -> np.ndarray:
    """Per-row data [modes*modes, N, m_max] of the sources f = sin(k pi x) sin(l pi y),
    k, l = 1..modes (row-major in (k, l)), g = 0: the right-hand side of a source with
    coefficients a is a @ basis (the learned warm start's inputs are these a)."""
    out = np.zeros((modes * modes, geom.n_sub, geom.m_max))
    for s in range(geom.n_sub):
        ri, _, _ = geom.rows(s)
        x, y = geom.xy[s, ri, 0], geom.xy[s, ri, 1]
        for k in range(modes):
            sx = np.sin((k + 1) * math.pi * x)
            for l in range(modes):
                out[k * modes + l, s, ri] = sx * np.sin((l + 1) * math.pi * y)
    return out


def test_points(geom: Geometry, n_side: int = 100):
    """n_side^2 cell-centred test points and the subdomain that owns each one
    (owner index min(floor(x*gx), gx-1) per axis)."""
    t = (np.arange(n_side, dtype=np.float64) + 0.5) / n_side
    X, Y = np.meshgrid(t, t, indexing="xy")
    xy = np.stack([X.ravel(), Y.ravel()], axis=1)
    ox = np.minimum((xy[:, 0] * geom.gx).astype(np.int64), geom.gx - 1)
    oy = np.minimum((xy[:, 1] * geom.gy).astype(np.int64), geom.gy - 1)
    return xy, (oy * geom.gx + ox).astype(np.int32)


# --------------------------------------------------------------------------
# Named workloads
# --------------------------------------------------------------------------

@dataclasses.dataclass
class Workload:
    name: str
    geom: Geometry
    n_neurons: int
    W: np.ndarray
    b: np.ndarray
    src: Source
    rhs: np.ndarray          # [N, m_max]
    test_xy: np.ndarray      # [T, 2]
    test_owner: np.ndarray   # [T]
    coef: Coefficient | None = None      # variable coefficient (None: -Laplacian)
    coef_rows: np.ndarray | None = None  # [N, m_max, 3]: rho, grad rho at every row


def build(gx, gy, n_neurons, mi_x, mi_y, p_bnd, p_ifc, theta="paper", theta_seed=0,
          source="sinsin", source_seed=0, modes=4, c=1.0 / 8.0, name="custom",
          n_test_side=100, m_max=None, coef=None, coef_seed=0, coef_alpha=16.0) -> Workload:
    """coef: None (-Laplacian) or a make_coefficient kind; with a coefficient the
    source's f becomes -div(rho grad u) of its closed-form u (or stays f = 1 for 'const')."""
    geom = make_geometry(gx, gy, mi_x, mi_y, p_bnd, p_ifc, m_max=m_max)
    W, b = draw_theta(geom, n_neurons, theta, theta_seed, c=c)
    src = make_source(source, source_seed, modes=modes)
    cf = None
    if coef is not None:
        cf = make_coefficient(coef, coef_seed, alpha=coef_alpha)
        src.params["coef"] = cf
    txy, own = test_points(geom, n_test_side)
    return Workload(name, geom, n_neurons, W, b, src, rhs_rows(geom, src), txy, own, cf,
                    coef_rows(geom, cf) if cf is not None else None)


def poisson_2x2_n200() -> Workload:
    """2x2 subdomains, 200 tanh neurons each, 20x20 interior points, 40 points per
    boundary and interface edge, u = sin(pi x) sin(pi y), theta ~ U(-1,1) (local
    coordinates), seed 1."""
    return build(2, 2, 200, 20, 20, 40, 40, theta="local_unit", theta_seed=1,
                 source="sinsin", name="poisson_2x2_n200")


def poisson_8x8_n1000() -> Workload:
    """8x8 subdomains, 1000 tanh neurons each, 50x40 interior points, 100 points per
    boundary and interface edge, f from 16 sine modes with N(0,1) coefficients
    (seed 2), paper initialisation c = 1/8 (seed 2)."""
    return build(8, 8, 1000, 50, 40, 100, 100, theta="paper", theta_seed=2,
                 source="fourier", source_seed=2, modes=4, name="poisson_8x8_n1000")


def poisson_16x16_n2000() -> Workload:
    """16x16 subdomains, 2000 neurons, 80x50 interior points, 128 points per edge."""
    return build(16, 16, 2000, 80, 50, 128, 128, theta="paper", theta_seed=3,
                 source="fourier", source_seed=3, modes=4, name="poisson_16x16_n2000")


def poisson_4x4_n1000() -> Workload:
    """4x4 subdomains with the per-subdomain shape of the 8x8 workload (1000 neurons,
    50x40 interior points, 100 points per edge): a smaller case of the same kernels."""
    return build(4, 4, 1000, 50, 40, 100, 100, theta="paper", theta_seed=2,
                 source="fourier", source_seed=2, modes=4, name="poisson_4x4_n1000")


def varcoef_4x4_n800() -> Workload:
    """-div(rho grad u) = f with rho = 1 + 0.5 sin(2 pi k . x), k_i uniform in {1..4}
    (seed 4); 4x4 subdomains, 800 neurons, 2 n_N interior points (40x40), 64 points per
    edge, manufactured u = sin(pi x) sin(pi y), paper initialisation (seed 4)."""
    return build(4, 4, 800, 40, 40, 64, 64, theta="paper", theta_seed=4, source="sinsin",
                 coef="sine", coef_seed=4, name="varcoef_4x4_n800")


def varcoef_grf_4x4_n800() -> Workload:
    """The paper's variable-coefficient problem: rho = tanh(grf) + 1.1 (alpha = 16,
    seed 6), f = 1, g = 0 (no closed form; its FEM reference is out of scope)."""
    return build(4, 4, 800, 40, 40, 64, 64, theta="paper", theta_seed=6, source="const",
                 coef="grf", coef_seed=6, name="varcoef_grf_4x4_n800")


def make_paper_grid_geometry(G: int, n_grid: int = 257, cross_points: bool = False) -> Geometry:
    """The paper's collocation layout (Section 4.2): the global uniform n_grid x n_grid grid
    of [0, 1]^2 split among G x G subdomains whose boundaries lie on grid lines.  Subdomain
    rows: its grid points strictly inside (interior), its grid points on the outer boundary
    (boundary; a point where an interface line meets the outer boundary is a boundary row
    of both subdomains), and the grid points strictly inside each of its interface edges
    (interface; one unknown per point, shared by the two subdomains of the edge).
    Interface unknowns are numbered edge by edge like make_geometry's (vertical edges
    first).

    The (G - 1)^2 cross points, where four subdomains meet, are left out unless
    ``cross_points``.  With them, each cross point is one more interface unknown (numbered
    after the edge unknowns, row by row), an interface row of each of its four
    subdomains, and the corner rule of the remark in Section 3 applies: A^s gets one row
    per edge through the point, with that edge's normal.  The rows of A^s are then given
    explicitly (``flux``): for every interface edge of s, its points and then its ends
    that are cross points (by increasing coordinate), all with the edge's outward normal;
    the flux conditions are numbered edge by edge in the same order."""
    h = n_grid - 1
    if h % G:
        raise ValueError("the grid lines must contain the subdomain boundaries")
    k = h // G                      # intervals per subdomain side
    t = np.arange(n_grid, dtype=np.float64) / h
    n_edge_dof = 2 * G * (G - 1) * (k - 1)
    n_edges = 2 * G * (G - 1)

    def vertex(X, Y):
        """Unknown of the cross point on grid lines (X, Y), or None."""
        if 1 <= X <= G - 1 and 1 <= Y <= G - 1:
            return n_edge_dof + (Y - 1) * (G - 1) + (X - 1)
        return None

    def edge_ends(ix, iy, e):
        """Cross points at the ends of edge e of subdomain (ix, iy), by increasing coordinate."""
        if e in ("left", "right"):
            X = ix + (1 if e == "right" else 0)
            ends = [(X, iy), (X, iy + 1)]
        else:
            Y = iy + (1 if e == "top" else 0)
            ends = [(ix, Y), (ix + 1, Y)]
        return [(XY, vertex(*XY)) for XY in ends if vertex(*XY) is not None]

    # flux conditions: edge by edge, its k - 1 points and then its cross-point ends
    f0 = np.zeros(n_edges + 1, np.int64)
    if cross_points:
        ends_of = {}
        for s in range(G * G):
            ix, iy = s % G, s // G
            for e in _EDGES:
                eid = _edge_id(G, G, ix, iy, e)
                if eid is not None:
                    ends_of[eid] = len(edge_ends(ix, iy, e))
        for eid in range(n_edges):
            f0[eid + 1] = f0[eid] + (k - 1) + ends_of[eid]
    per = []
    for s in range(G * G):
        ix, iy = s % G, s // G
        xs, ys = t[ix * k:(ix + 1) * k + 1], t[iy * k:(iy + 1) * k + 1]   # k + 1 lines each
        X, Y = np.meshgrid(xs[1:-1], ys[1:-1], indexing="xy")
        interior = np.stack([X.ravel(), Y.ravel()], axis=1)
        bnd = []
        if iy == 0:
            bnd.append(np.stack([xs, np.zeros(k + 1)], axis=1))
        if iy == G - 1:
            bnd.append(np.stack([xs, np.ones(k + 1)], axis=1))
        if ix == 0:
            bnd.append(np.stack([np.zeros(k + 1), ys], axis=1))
        if ix == G - 1:
            bnd.append(np.stack([np.ones(k + 1), ys], axis=1))
        bnd = np.unique(np.concatenate(bnd), axis=0) if bnd else np.zeros((0, 2))
        ifc, nrm, dof = [], [], []
        frow, fnrm, fdof = [], [], []
        corners = {}                # cross-point unknown -> its interface row in s
        if cross_points:
            nedge_rows = (k - 1) * sum(_edge_id(G, G, ix, iy, e) is not None for e in _EDGES)
            for XY in [(ix, iy), (ix + 1, iy), (ix, iy + 1), (ix + 1, iy + 1)]:
                v = vertex(*XY)
                if v is not None:
                    corners[v] = nedge_rows + len(corners)
        nrow = 0
        for e in _EDGES:
            eid = _edge_id(G, G, ix, iy, e)
            if eid is None:
                continue
            if e in ("left", "right"):
                xe = t[(ix + (1 if e == "right" else 0)) * k]
                pts = np.stack([np.full(k - 1, xe), t[iy * k + 1:(iy + 1) * k]], axis=1)
            else:
                ye = t[(iy + (1 if e == "top" else 0)) * k]
                pts = np.stack([t[ix * k + 1:(ix + 1) * k], np.full(k - 1, ye)], axis=1)
            ifc.append(pts)
            nrm.append(np.tile(np.array(_NORMALS[e]), (k - 1, 1)))
            dof.append(eid * (k - 1) + np.arange(k - 1))
            if cross_points:
                ends = edge_ends(ix, iy, e)
                frow += list(range(nrow, nrow + k - 1)) + [corners[v] for _, v in ends]
                fnrm += [_NORMALS[e]] * (k - 1 + len(ends))
                fdof += list(range(f0[eid], f0[eid + 1]))
            nrow += k - 1
        for v, r in corners.items():
            X, Y = (v - n_edge_dof) % (G - 1) + 1, (v - n_edge_dof) // (G - 1) + 1
            ifc.append(np.array([[t[X * k], t[Y * k]]]))
            nrm.append(np.zeros((1, 2)))      # its A^s rows are the flux rows above
            dof.append(np.array([v]))
        ifc = np.concatenate(ifc) if ifc else np.zeros((0, 2))
        nrm = np.concatenate(nrm) if nrm else np.zeros((0, 2))
        dof = np.concatenate(dof).astype(np.int32) if dof else np.zeros(0, np.int32)
        per.append((interior, bnd, ifc, nrm, dof, (frow, fnrm, fdof)))
    m_max = max(len(a) + len(b) + len(c) for a, b, c, _, _, _ in per)
    N = G * G
    counts = np.zeros((N, 3), np.int32)
    xy = np.zeros((N, m_max, 2))
    nr = np.zeros((N, m_max, 2))
    dd = np.full((N, m_max), -1, np.int32)
    for s, (interior, bnd, ifc, nrm, dof, _) in enumerate(per):
        mi, mb, mg = len(interior), len(bnd), len(ifc)
        counts[s] = (mi, mb, mg)
        xy[s, :mi] = interior
        xy[s, mi:mi + mb] = bnd
        xy[s, mi + mb:mi + mb + mg] = ifc
        nr[s, mi + mb:mi + mb + mg] = nrm
        dd[s, mi + mb:mi + mb + mg] = dof
    n_gamma = n_edge_dof + ((G - 1) ** 2 if cross_points else 0)
    flux = None
    if cross_points:
        f_max = max(len(f[0]) for *_, f in per)
        fc = np.zeros(N, np.int32)
        fr = np.zeros((N, f_max), np.int32)
        fn = np.zeros((N, f_max, 2))
        fd = np.full((N, f_max), -1, np.int32)
        for s, (*_, (frow, fnrm, fdof)) in enumerate(per):
            fc[s] = len(frow)
            fr[s, :len(frow)] = frow
            fn[s, :len(frow)] = np.array(fnrm).reshape(-1, 2)
            fd[s, :len(frow)] = fdof
        flux = FluxRows(int(f0[-1]), fc, fr, fn, fd)
    return Geometry(G, G, k - 1, k - 1, k + 1, k - 1, counts, xy, nr, dd, n_gamma, flux)


def paper_grid_workload(G: int, n_total: int = 65536, theta: str = "paper", seed: int = 0,
                        source: str = "sin2pi_exp", n_grid: int = 257, n_test_side: int = 100,
                        cross_points: bool = False) -> Workload:
    """The paper's Poisson experiments (Section 4.2, Table 2; Table 1 with other theta
    modes): n_total neurons split evenly over G x G subdomains, the global n_grid^2
    collocation grid (make_paper_grid_geometry, with or without its cross points),
    u = sin(2 pi x) e^y by default, theta by Eq. (4.3) with c = 1/8 (``paper``), or
    ``global_unit`` (Table 1's manual l = 1) or ``he`` (Table 1's He initialisation)."""
    geom = make_paper_grid_geometry(G, n_grid, cross_points)
    n = n_total // (G * G)
    W, b = draw_theta(geom, n, theta, seed, c=1.0 / 8.0)
    src = make_source(source, seed)
    txy, own = test_points(geom, n_test_side)
    name = f"paper_grid_{G}x{G}_{theta}" + ("_cross" if cross_points else "")
    return Workload(name, geom, n, W, b, src, rhs_rows(geom, src), txy, own)


def mixed_16x16_n60_local() -> Workload:
    """16 x 16 subdomains with few neurons (60, 40 x 40 interior points, 40 points per edge) and
    local U(-1, 1) weights: kappa(K^s) ~ 1e6, well-conditioned enough for the mixed-precision
    path to refine instead of falling back (the 16 x 16 decomposition of the mixed-precision
    configuration with a network small enough to be well conditioned)."""
    return build(16, 16, 60, 40, 40, 40, 40, theta="local_unit", theta_seed=16, source="fourier",
                 source_seed=16, modes=4, name="mixed_16x16_n60_local")


WORKLOADS = {
    "paper_grid_4x4": lambda: paper_grid_workload(4, seed=41),
    "paper_grid_8x8": lambda: paper_grid_workload(8, seed=81),
    "paper_grid_16x16": lambda: paper_grid_workload(16, seed=161),
    "mixed_16x16_n60_local": mixed_16x16_n60_local,
    "varcoef_4x4_n800": varcoef_4x4_n800,
    "varcoef_grf_4x4_n800": varcoef_grf_4x4_n800,
    "poisson_2x2_n200": poisson_2x2_n200,
    "poisson_4x4_n1000": poisson_4x4_n1000,
    "poisson_8x8_n1000": poisson_8x8_n1000,
    "poisson_16x16_n2000": poisson_16x16_n2000,
}
