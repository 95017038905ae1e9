"""Sim(3) pose-graph optimisation: the oracle (Sec. III-E of the paper).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Nodes are submap poses T_t in Sim(3) (submap -> world).  An edge (i, j)
carries the relative transform T_ij from registration, and its error is

    e_ij = log_Sim3(T_ij^-1 T_i^-1 T_j),

which vanishes when T_j = T_i T_ij.  The energy is
chi^2 = sum_(i,j) e_ij^T Omega_ij e_ij.  The poses are initialised by
chaining the relative transforms and then optimised.

Readings (the paper names Levenberg-Marquardt in PyPose and no more):

* Gauss-Newton with right perturbations T <- T Exp(delta), ``iters``
  iterations, optional damping H + lambda I (``lm_lambda`` > 0);
* node ``fixed`` (default 0) is held constant to fix the gauge;
* Omega_ij = I_7 unless given;
* chaining initialisation walks a spanning tree made of the edges, taken in
  input order, that join two not-yet-connected parts of the graph (for an
  odometry chain listed first this is the chain itself), outward from the
  fixed node: T_j = T_i T_ij along an edge, T_i = T_j T_ij^-1 against it;
* Jacobians are central finite differences in float64 of the edge error
  itself, with one Richardson extrapolation step, and the normal equations are solved by a dense
  Cholesky factorisation (``numpy.linalg.cholesky``).
"""
from __future__ import annotations

from collections import deque

import numpy as np

from . import sim3


def edge_error(Ti, Tj, Tij):
    return sim3.log(sim3.compose(sim3.inverse(Tij), sim3.compose(sim3.inverse(Ti), Tj)))


def chi2(nodes, ei, ej, Tij, info=None):
    tot = 0.0
    for k in range(len(ei)):
        e = edge_error(nodes[ei[k]], nodes[ej[k]], Tij[k])
        Om = np.eye(7) if info is None else np.asarray(info[k]).reshape(7, 7)
        tot += float(e @ Om @ e)
    return tot


def spanning_tree(n, ei, ej):
    """Edges (in input order) that join two different components."""
    parent = list(range(n))

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a

    tree = []
    for k in range(len(ei)):
        a, b = find(int(ei[k])), find(int(ej[k]))
        if a != b:
            parent[a] = b
            tree.append(k)
    return tree


def chain_init(n, ei, ej, Tij, root=0, T_root=None):
    """Poses from chaining relative transforms along the spanning tree."""
    adj = [[] for _ in range(n)]
    for k in spanning_tree(n, ei, ej):
        adj[int(ei[k])].append(k)
        adj[int(ej[k])].append(k)
    nodes = [None] * n
    nodes[root] = sim3.identity() if T_root is None else T_root
    dq = deque([root])
    while dq:
        a = dq.popleft()
        for k in adj[a]:
            i, j = int(ei[k]), int(ej[k])
            if a == i and nodes[j] is None:
                nodes[j] = sim3.compose(nodes[i], Tij[k])
                dq.append(j)
            elif a == j and nodes[i] is None:
                nodes[i] = sim3.compose(nodes[j], sim3.inverse(Tij[k]))
                dq.append(i)
    for v in range(n):
        if nodes[v] is None:           # not connected to the root: identity
            nodes[v] = sim3.identity()
    return nodes


def numeric_jacobians(Ti, Tj, Tij, h=1e-3):
    """d e_ij / d delta for T_i <- T_i Exp(delta_i) and T_j <- T_j Exp(delta_j).

    Central differences with one Richardson extrapolation step,
    (4 D(h/2) - D(h)) / 3, whose truncation error is O(h^4).
    """
    def central(which, a, step):
        d = np.zeros(7)
        d[a] = step
        if which == 0:
            ep = edge_error(sim3.compose(Ti, sim3.exp(d)), Tj, Tij)
            em = edge_error(sim3.compose(Ti, sim3.exp(-d)), Tj, Tij)
        else:
            ep = edge_error(Ti, sim3.compose(Tj, sim3.exp(d)), Tij)
            em = edge_error(Ti, sim3.compose(Tj, sim3.exp(-d)), Tij)
        return (ep - em) / (2 * step)

    Ji = np.zeros((7, 7))
    Jj = np.zeros((7, 7))
    for a in range(7):
        Ji[:, a] = (4 * central(0, a, h / 2) - central(0, a, h)) / 3
        Jj[:, a] = (4 * central(1, a, h / 2) - central(1, a, h)) / 3
    return Ji, Jj


def normal_equations(nodes, ei, ej, Tij, info, fixed, h=1e-3):
    """H = sum J^T Omega J and g = sum J^T Omega e over the free nodes."""
    n = len(nodes)
    free = [v for v in range(n) if v != fixed]
    col = {v: 7 * q for q, v in enumerate(free)}
    H = np.zeros((7 * len(free), 7 * len(free)))
    g = np.zeros(7 * len(free))
    for k in range(len(ei)):
        i, j = int(ei[k]), int(ej[k])
        e = edge_error(nodes[i], nodes[j], Tij[k])
        Ji, Jj = numeric_jacobians(nodes[i], nodes[j], Tij[k], h)
        Om = np.eye(7) if info is None else np.asarray(info[k]).reshape(7, 7)
        for a, Ja in ((i, Ji), (j, Jj)):
            if a == fixed:
                continue
            g[col[a]:col[a] + 7] += Ja.T @ Om @ e
            for b, Jb in ((i, Ji), (j, Jj)):
                if b == fixed:
                    continue
                H[col[a]:col[a] + 7, col[b]:col[b] + 7] += Ja.T @ Om @ Jb
    return H, g, free, col


LM_MIN, LM_MAX = 1e-10, 1e10


def levenberg_marquardt(nodes, ei, ej, Tij, info=None, iters=10, fixed=0, lambda0=1e-3,
                        h=1e-3):
    """Levenberg-Marquardt (Sec. III-E: the paper optimises with LM): each step
    solves (H + lambda I) delta = -g; it is kept when the Cholesky
    factorisation exists and chi^2 decreases (lambda / 10, not below 1e-10),
    else discarded (lambda x 10, not above 1e10).

    Returns (nodes, chi2 history of length iters+1: before each step and after
    the last, lambdas used)."""
    nodes = list(nodes)
    lam = float(lambda0)
    hist = [chi2(nodes, ei, ej, Tij, info)]
    lams = []
    for _ in range(iters):
        lams.append(lam)
        H, g, free, col = normal_equations(nodes, ei, ej, Tij, info, fixed, h)
        trial = None
        try:
            L = np.linalg.cholesky(H + lam * np.eye(H.shape[0]))
            delta = np.linalg.solve(L.T, np.linalg.solve(L, -g))
            trial = list(nodes)
            for v in free:
                trial[v] = sim3.compose(nodes[v], sim3.exp(delta[col[v]:col[v] + 7]))
        except np.linalg.LinAlgError:
            pass
        if trial is not None and chi2(trial, ei, ej, Tij, info) < hist[-1]:
            nodes = trial
            lam = max(lam * 0.1, LM_MIN)
        else:
            lam = min(lam * 10.0, LM_MAX)
        hist.append(chi2(nodes, ei, ej, Tij, info))
    return nodes, hist, lams


def gauss_newton(nodes, ei, ej, Tij, info=None, iters=10, fixed=0, lm_lambda=0.0, h=1e-3):
    """Returns (nodes, chi2 history of length iters+1, last step norms)."""
    n = len(nodes)
    nodes = list(nodes)
    hist = [chi2(nodes, ei, ej, Tij, info)]
    steps = []
    free = [v for v in range(n) if v != fixed]
    col = {v: 7 * q for q, v in enumerate(free)}
    for _ in range(iters):
        H = np.zeros((7 * len(free), 7 * len(free)))
        g = np.zeros(7 * len(free))
        for k in range(len(ei)):
            i, j = int(ei[k]), int(ej[k])
            e = edge_error(nodes[i], nodes[j], Tij[k])
            Ji, Jj = numeric_jacobians(nodes[i], nodes[j], Tij[k], h)
            Om = np.eye(7) if info is None else np.asarray(info[k]).reshape(7, 7)
            for a, Ja in ((i, Ji), (j, Jj)):
                if a == fixed:
                    continue
                g[col[a]:col[a] + 7] += Ja.T @ Om @ e
                for b, Jb in ((i, Ji), (j, Jj)):
                    if b == fixed:
                        continue
                    H[col[a]:col[a] + 7, col[b]:col[b] + 7] += Ja.T @ Om @ Jb
        if lm_lambda > 0:
            H = H + lm_lambda * np.eye(H.shape[0])
        L = np.linalg.cholesky(H)
        y = np.linalg.solve(L, -g)
        delta = np.linalg.solve(L.T, y)
        for v in free:
            nodes[v] = sim3.compose(nodes[v], sim3.exp(delta[col[v]:col[v] + 7]))
        steps.append(float(np.linalg.norm(delta)))
        hist.append(chi2(nodes, ei, ej, Tij, info))
    return nodes, hist, steps
