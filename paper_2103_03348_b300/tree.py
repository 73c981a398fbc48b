"""The phylogenetic Brownian prior on the sequenced log-rates (Section 2.2,
Eq. 2) evaluated in O(M) on the tree (Section 2.3.1's dynamic programme),
through the library's hawkes_tree_plan (host) and hawkes_tree_prior (device).

Tree encoding: nodes 0..M-1 are the tips in the order of the sequenced events;
nodes M..2M-2 are internal; parent[v] is -1 at the root; length[v] is the
branch length from v to its parent.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import hawkes


def _lib():
    L = hawkes.lib()
    if not getattr(L, "_tree_typed", False):
        vp, i64, d, sz = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_size_t
        L.hawkes_tree_plan_size.argtypes = [i64]
        L.hawkes_tree_plan_size.restype = sz
        L.hawkes_tree_workspace_size.argtypes = [i64]
        L.hawkes_tree_workspace_size.restype = sz
        L.hawkes_tree_plan.argtypes = [i64, vp, vp, sz]
        L.hawkes_tree_plan.restype = ctypes.c_int
        L.hawkes_tree_prior.argtypes = [i64, vp, vp, d, d, vp, vp, sz, vp, vp, vp, vp]
        L.hawkes_tree_prior.restype = ctypes.c_int
        L.hawkes_posterior_tree_workspace_size.argtypes = [i64]
        L.hawkes_posterior_tree_workspace_size.restype = sz
        L.hawkes_tree_mass_workspace_size.argtypes = [i64]
        L.hawkes_tree_mass_workspace_size.restype = sz
        L.hawkes_tree_mass_factor.argtypes = [i64, vp, vp, d, d, vp, vp, vp, sz, vp]
        L.hawkes_tree_mass_factor.restype = ctypes.c_int
        L.hawkes_tree_mass_velocity.argtypes = [i64, vp, vp, i64, vp, i64, i64, vp, vp, vp, vp, d, vp, vp, sz, vp]
        L.hawkes_tree_mass_velocity.restype = ctypes.c_int
        L.hawkes_tree_mass_momentum.argtypes = [i64, vp, vp, d, d, vp, i64, vp, i64, i64, vp, vp, vp, vp, sz, vp]
        L.hawkes_tree_mass_momentum.restype = ctypes.c_int
        L._tree_typed = True
    return L


def _check(rc):
    if rc != hawkes.OK:
        raise hawkes.HawkesError(rc, hawkes.strerror(rc))


def plan(parent) -> np.ndarray:
    """The host traversal plan (int32) for a parent array of 2M-1 nodes."""
    L = _lib()
    par = np.ascontiguousarray(parent, dtype=np.int64)
    nn = par.size
    if nn < 3 or nn % 2 == 0:
        raise hawkes.HawkesError(hawkes.EINVAL, "parent must have 2M-1 entries with M >= 2")
    m = (nn + 1) // 2
    size = int(L.hawkes_tree_plan_size(m))
    if size == 0:
        raise hawkes.HawkesError(hawkes.EINVAL, "tree too large")
    out = np.zeros(size // 4, dtype=np.int32)
    _check(L.hawkes_tree_plan(m, par.ctypes.data_as(ctypes.c_void_p), out.ctypes.data_as(ctypes.c_void_p),
                              ctypes.c_size_t(size)))
    return out


class TreePrior:
    """z ~ N(0, sigma2 V) with V from the tree; plan and branch lengths live on the device."""

    def __init__(self, parent, length, root_var: float, sigma2: float, device="cuda"):
        self.parent = np.asarray(parent, dtype=np.int64)
        self.m = (self.parent.size + 1) // 2
        host_plan = plan(self.parent)
        self.plan = torch.from_numpy(host_plan).to(device)
        self.length = torch.as_tensor(np.asarray(length, dtype=np.float64), device=device).contiguous()
        if self.length.numel() != self.parent.size:
            raise hawkes.HawkesError(hawkes.EINVAL, "length must have 2M-1 entries")
        self.root_var = float(root_var)
        self.sigma2 = float(sigma2)
        self.levels = int(host_plan[0])
        self.ws = torch.empty(int(_lib().hawkes_tree_workspace_size(self.m)), dtype=torch.uint8, device=device)

    def evaluate(self, z, want=("logdens", "pz", "pdiag"), out=None):
        """{'logdens': log N(z; 0, sigma2 V), 'pz': (sigma2 V)^-1 z, 'pdiag': diag((sigma2 V)^-1)}.

        out: optional dict of preallocated device tensors (a missing or None
        entry is not computed); enqueued on the current stream."""
        L = _lib()
        z = z.contiguous()
        f64 = dict(dtype=torch.float64, device=z.device)
        if out is None:
            out = {"logdens": torch.empty((), **f64) if "logdens" in want else None,
                   "pz": torch.empty(self.m, **f64) if "pz" in want else None,
                   "pdiag": torch.empty(self.m, **f64) if "pdiag" in want else None}
        else:
            out = {k: out.get(k) for k in ("logdens", "pz", "pdiag")}
        p = lambda t: ctypes.c_void_p(t.data_ptr() if t is not None else 0)  # noqa: E731
        s = ctypes.c_void_p(torch.cuda.current_stream(z.device).cuda_stream)
        _check(L.hawkes_tree_prior(self.m, p(self.plan), p(self.length), self.root_var, self.sigma2, p(z), p(self.ws),
                                   ctypes.c_size_t(self.ws.numel()), p(out["logdens"]), p(out["pz"]),
                                   p(out["pdiag"]), s))
        return {k: v for k, v in out.items() if v is not None}


class TreeMass:
    """The HMC mass matrix with the phylogenetic prior's full precision on the
    rate block: M = diag(1 / minv) outside coordinates [z0, z0 + m) of a
    k-dimensional state, M_z = diag(d) + (sigma2 V)^-1 on them, d >= 0 the
    likelihood's curvature (self.d, a device tensor the caller updates in
    place, calling factor() after each change).  Every call is a tree sweep
    on the device (O(m), no M x M matrix), enqueued on the current stream.

    nc > 0 couples the first nc coordinates with the rate block through
    set_coupling(A, B): M = [[A, B^T], [B, M_z]] (see hawkes.h)."""

    def __init__(self, prior: TreePrior, k: int, z0: int = 6, nc: int = 0):
        if z0 < 0 or z0 + prior.m > k:
            raise hawkes.HawkesError(hawkes.EINVAL, "the rate block must lie inside the state")
        self.prior, self.k, self.z0, self.m = prior, int(k), int(z0), prior.m
        dev = prior.length.device
        self.d = torch.zeros(self.m, dtype=torch.float64, device=dev)
        self.fac = torch.empty(2 * (2 * self.m - 1), dtype=torch.float64, device=dev)
        self.ws = torch.empty(int(_lib().hawkes_tree_mass_workspace_size(self.m)), dtype=torch.uint8, device=dev)
        self.n_normals = self.k + 2 * self.m - 1
        if not 0 <= nc <= min(self.z0, 8):
            raise hawkes.HawkesError(hawkes.EINVAL, "at most 8 coupled coordinates, all before the rate block")
        self.nc = int(nc)
        self.cpl = torch.zeros(max(1, self.m * self.nc + 2 * self.nc * self.nc), dtype=torch.float64, device=dev)
        self.coupling_shrink = 1.0

    def set_coupling(self, A, B, floor=1e-2):
        """Couple the first nc coordinates to the rate block with the mass
        blocks A (nc x nc) and B (m x nc) (host arrays), for the current d
        (call factor() first).  A is made positive definite by clipping its
        eigenvalues at floor; B is shrunk by a factor c <= 1 where needed so
        that S = A - c^2 B^T M_z^-1 B keeps at least a tenth of A's curvature
        in every direction (self.coupling_shrink = c).  Small host algebra on
        nc x nc matrices; U = M_z^-1 B comes from nc velocity sweeps."""
        nc, m = self.nc, self.m
        A = np.asarray(A, float).reshape(nc, nc)
        B = np.asarray(B, float).reshape(m, nc)
        w, Q = np.linalg.eigh(0.5 * (A + A.T))
        A = (Q * np.maximum(w, floor)) @ Q.T
        dev = self.d.device
        U = np.empty((m, nc))
        minv = torch.ones(self.k, dtype=torch.float64, device=dev)
        vel = torch.empty(self.k, dtype=torch.float64, device=dev)
        pb = torch.zeros(self.k, dtype=torch.float64, device=dev)
        saved, self.nc = self.nc, 0  # the sweeps for U use the uncoupled mass
        try:
            for j in range(nc):
                pb[self.z0:self.z0 + m] = torch.as_tensor(B[:, j], device=dev)
                self.velocity(pb, minv, vel=vel)
                U[:, j] = vel[self.z0:self.z0 + m].cpu().numpy()
        finally:
            self.nc = saved
        G = B.T @ U
        G = 0.5 * (G + G.T)
        wa, Qa = np.linalg.eigh(A)
        ih = (Qa / np.sqrt(wa)) @ Qa.T  # A^-1/2
        lam = float(np.linalg.eigvalsh(ih @ G @ ih).max())
        c = 1.0 if lam <= 0.9 else float(np.sqrt(0.9 / lam))
        S = A - c * c * G
        S = 0.5 * (S + S.T)
        Lc = np.linalg.cholesky(S)
        buf = np.concatenate([(c * U).ravel(), np.linalg.inv(S).ravel(), Lc.ravel()])
        self.cpl[:buf.size].copy_(torch.as_tensor(buf, device=dev))
        self.coupling_shrink = c

    def factor(self):
        """The sweep coefficients for the current self.d (call after changing it)."""
        t = lambda a: ctypes.c_void_p(a.data_ptr())  # noqa: E731
        s = ctypes.c_void_p(torch.cuda.current_stream(self.d.device).cuda_stream)
        pr = self.prior
        _check(_lib().hawkes_tree_mass_factor(self.m, t(pr.plan), t(pr.length), pr.root_var, pr.sigma2, t(self.d),
                                              t(self.fac), t(self.ws), ctypes.c_size_t(self.ws.numel()), s))

    def velocity(self, p, minv, vel=None, q=None, eps=0.0, kinetic=None):
        """vel = M^-1 p; q += eps M^-1 p; kinetic = p^T M^-1 p / 2 (each when given)."""
        t = lambda a: ctypes.c_void_p(a.data_ptr() if a is not None else 0)  # noqa: E731
        s = ctypes.c_void_p(torch.cuda.current_stream(p.device).cuda_stream)
        _check(_lib().hawkes_tree_mass_velocity(self.m, t(self.prior.plan), t(self.fac), self.nc, t(self.cpl), self.k,
                                                self.z0, t(minv), t(p), t(vel), t(q), float(eps), t(kinetic),
                                                t(self.ws), ctypes.c_size_t(self.ws.numel()), s))

    def momentum(self, minv, xi, p):
        """p ~ N(0, M) from xi, k + 2m - 1 standard normals (device)."""
        if xi.numel() != self.n_normals or p.numel() != self.k:
            raise hawkes.HawkesError(hawkes.EINVAL, "xi must hold k + 2m - 1 normals and p k entries")
        t = lambda a: ctypes.c_void_p(a.data_ptr())  # noqa: E731
        s = ctypes.c_void_p(torch.cuda.current_stream(p.device).cuda_stream)
        pr = self.prior
        _check(_lib().hawkes_tree_mass_momentum(self.m, t(pr.plan), t(pr.length), pr.root_var, pr.sigma2, t(self.d),
                                                self.nc, t(self.cpl), self.k, self.z0, t(minv), t(xi), t(p),
                                                t(self.ws), ctypes.c_size_t(self.ws.numel()), s))
        return p
