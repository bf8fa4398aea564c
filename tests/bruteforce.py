"""A second, deliberately different evaluation of the residual and sensor, used only to
pin the oracle on tiny meshes.

It works from the same definitions (Eq. weak2, the LLF flux of Sec. 2, the stabilization
of Sec. 3 and the sensor of Sec. 4) but shares no code with the oracle: Legendre
polynomials come from NumPy's ``numpy.polynomial.legendre`` (Clenshaw evaluation,
``legder`` for derivatives), every integral uses a 24-point Gauss rule in physical
coordinates, the wave speed s+ is a maximum over a dense sample of the segment
including its end points (exact for the linear and Burgers fluxes used here), and the
mass matrix is the closed form (h/2)^d prod 2/(2i+1).
"""
from __future__ import annotations

import numpy as np
from numpy.polynomial import legendre as npleg

NQ = 24
_g, _w = npleg.leggauss(NQ)


def _P(n, a, x):
    c = np.zeros(n + 1)
    c[n] = 1.0
    if a:
        c = npleg.legder(c, a)
    return npleg.legval(x, c)


class Mesh:
    def __init__(self, P):
        self.P = P
        self.h = (P.box[1] - P.box[0]) / P.nx
        self.n1 = P.p + 1

    def centre(self, e):
        P = self.P
        ix, iy = e % P.nx, e // P.nx
        xc = P.box[0] + (ix + 0.5) * self.h
        yc = P.box[2] + (iy + 0.5) * self.h if P.dim == 2 else 0.0
        return xc, yc

    def basis(self, k, kx, ky, c, x, y):
        """Physical derivative D^(kx,ky) of phi_k of the element centred at c."""
        i, j = k % self.n1, k // self.n1
        v = _P(i, kx, 2 * (x - c[0]) / self.h) * (2 / self.h) ** kx
        if self.P.dim == 2:
            v = v * _P(j, ky, 2 * (y - c[1]) / self.h) * (2 / self.h) ** ky
        return v

    def poly(self, coef, kx, ky, c, x, y):
        return sum(coef[k] * self.basis(k, kx, ky, c, x, y) for k in range(len(coef)))

    def vol_pts(self, e):
        xc, yc = self.centre(e)
        if self.P.dim == 1:
            return xc + 0.5 * self.h * _g, np.zeros(NQ), 0.5 * self.h * _w
        X, Y = np.meshgrid(xc + 0.5 * self.h * _g, yc + 0.5 * self.h * _g, indexing="xy")
        W = np.outer(_w, _w) * 0.25 * self.h ** 2
        return X.ravel(), Y.ravel(), W.ravel()

    def nbr(self, e, f):
        P = self.P
        ix, iy = e % P.nx, e // P.nx
        d = [(-1, 0), (1, 0), (0, -1), (0, 1)][f]
        jx, jy = ix + d[0], iy + d[1]
        xc, yc = self.centre(e)
        c = (xc + d[0] * self.h, yc + d[1] * self.h)
        if not (0 <= jx < P.nx):
            if P.bc[f] != "periodic":
                return None, c
            jx %= P.nx
        if P.dim == 2 and not (0 <= jy < P.ny):
            if P.bc[f] != "periodic":
                return None, c
            jy %= P.ny
        return jy * P.nx + jx, c


def _flux(P, u, x, y):
    if P.flux == "advect":
        F = (P.a[0] * u, P.a[1] * u)
    elif P.flux == "rotation":
        F = (P.omega * (P.center[1] - y) * u, P.omega * (x - P.center[0]) * u)
    elif P.flux == "burgers":
        F = (P.a[0] * 0.5 * u * u, P.a[1] * 0.5 * u * u)
    else:
        raise ValueError(P.flux)
    return F if P.dim == 2 else (F[0], 0.0 * F[1])


def _dflux(P, u, x, y):
    if P.flux == "advect":
        v = (P.a[0] + 0 * u, P.a[1] + 0 * u)
    elif P.flux == "rotation":
        v = (P.omega * (P.center[1] - y) + 0 * u, P.omega * (x - P.center[0]) + 0 * u)
    elif P.flux == "burgers":
        v = (P.a[0] * u, P.a[1] * u)
    else:
        raise ValueError(P.flux)
    return v if P.dim == 2 else (v[0], 0.0 * v[1])


def _llf(P, um, up, x, y, n):
    Fm, Fp = _flux(P, um, x, y), _flux(P, up, x, y)
    om = np.linspace(0.0, 1.0, 2001)[:, None]
    uw = om * um[None, :] + (1 - om) * up[None, :]
    v = _dflux(P, uw, x[None, :], y[None, :])
    s = np.max(np.abs(v[0] * n[0] + v[1] * n[1]), axis=0)
    return 0.5 * (n[0] * (Fm[0] + Fp[0]) + n[1] * (Fm[1] + Fp[1])) - 0.5 * s * (up - um)


def _seminorm2(m, coef, c):
    P = m.P
    X, Y, W = m.vol_pts(0)
    c0 = m.centre(0)
    X, Y = X - c0[0] + c[0], Y - c0[1] + c[1]
    s = 0.0
    for ky in range(P.p + 1 if P.dim == 2 else 1):
        for kx in range(P.p + 1):
            K = kx + ky
            if 1 <= K <= P.p:
                d = m.poly(coef, kx, ky, c, X, Y)
                s += m.h ** (2 * K - P.dim) * np.sum(W * d * d)
    return s


def sensor(P, U):
    m = Mesh(P)
    E, K = P.E, P.K
    gam = np.zeros(E)
    for e in range(E):
        c = m.centre(e)
        ce = U[:, e]
        X, Y, W = m.vol_pts(e)
        cands = [ce.copy()]
        for f in range(2 * P.dim):
            nb, cn = m.nbr(e, f)
            if nb is None:
                continue
            vals = m.poly(U[:, nb], 0, 0, cn, X, Y)
            cl = np.array([np.sum(W * vals * m.basis(k, 0, 0, c, X, Y)) /
                           np.sum(W * m.basis(k, 0, 0, c, X, Y) ** 2) for k in range(K)])
            cl[0] = ce[0]
            cands.append(cl)
        me = len(cands) - 1
        lin = np.array([1 - me * P.w_nbr] + [P.w_nbr] * me)
        beta = np.array([_seminorm2(m, cl, c) for cl in cands])
        wt = lin / (P.eps_w + beta) ** 2
        w = wt / wt.sum()
        if P.stab == "zhao":
            # Zhao et al.'s sensor as restated in Sec. 5.6 (no neighbour: weights = linear)
            gam[e] = 0.0 if me == 0 else (np.sum(np.abs(w / lin - 1) ** P.theta) /
                                          (abs(1 / lin.min() - 1) ** P.theta + me))
            continue
        ustar = sum(wl * cl for wl, cl in zip(w, cands))
        num = np.sqrt(_seminorm2(m, ce - ustar, c))
        den = np.sqrt(_seminorm2(m, ce, c))
        if num <= P.eps_s:
            g = 0.0
        elif den == 0:
            g = 1.0
        else:
            r = num / den
            g = min(1.0, r) ** P.q
            if r < P.b:
                g = 0.0
        gam[e] = g
    return gam


def _lambda(P, m, e, ce):
    if P.lambda_nu > 0:
        return P.lambda_nu
    g, _ = npleg.leggauss(P.p + 2)
    xc, yc = m.centre(e)
    pts = []
    if P.dim == 1:
        pts = [(xc + 0.5 * m.h * t, 0.0) for t in g] + [(xc - 0.5 * m.h, 0.0), (xc + 0.5 * m.h, 0.0)]
    else:
        pts = [(xc + 0.5 * m.h * a, yc + 0.5 * m.h * b) for a in g for b in g]
        for s in (-1, 1):
            pts += [(xc + 0.5 * m.h * s, yc + 0.5 * m.h * t) for t in g]
            pts += [(xc + 0.5 * m.h * t, yc + 0.5 * m.h * s) for t in g]
    x = np.array([q[0] for q in pts])
    y = np.array([q[1] for q in pts])
    u = m.poly(ce, 0, 0, (xc, yc), x, y)
    v = _dflux(P, u, x, y)
    return float(np.max(np.sqrt(v[0] ** 2 + v[1] ** 2)))


def residual(P, U):
    m = Mesh(P)
    E, K = P.E, P.K
    L = np.zeros((K, E))
    gam = sensor(P, U) if P.stab in ("weno", "zhao") else np.full(E, 1.0 if P.stab == "lo" else 0.0)
    for e in range(E):
        c = m.centre(e)
        ce = U[:, e]
        X, Y, W = m.vol_pts(e)
        u = m.poly(ce, 0, 0, c, X, Y)
        F = _flux(P, u, X, Y)
        R = np.zeros(K)
        for k in range(K):
            R[k] = np.sum(W * m.basis(k, 1, 0, c, X, Y) * F[0])
            if P.dim == 2:
                R[k] += np.sum(W * m.basis(k, 0, 1, c, X, Y) * F[1])
        for f in range(2 * P.dim):
            n = [(-1.0, 0.0), (1.0, 0.0), (0.0, -1.0), (0.0, 1.0)][f]
            if P.dim == 1:
                fx = np.array([c[0] + 0.5 * m.h * n[0]])
                fy = np.zeros(1)
                fw = np.ones(1)
            elif f < 2:
                fx = np.full(NQ, c[0] + 0.5 * m.h * n[0])
                fy = c[1] + 0.5 * m.h * _g
                fw = 0.5 * m.h * _w
            else:
                fx = c[0] + 0.5 * m.h * _g
                fy = np.full(NQ, c[1] + 0.5 * m.h * n[1])
                fw = 0.5 * m.h * _w
            um = m.poly(ce, 0, 0, c, fx, fy)
            nb, cn = m.nbr(e, f)
            if nb is not None:
                up = m.poly(U[:, nb], 0, 0, cn, fx, fy)
            elif P.bc[f] == "inflow_zero":
                v = _dflux(P, um, fx, fy)
                up = np.where(v[0] * n[0] + v[1] * n[1] < 0, 0.0, um)
            else:
                up = um.copy()
            H = _llf(P, um, up, fx, fy, n)
            for k in range(K):
                R[k] -= np.sum(fw * m.basis(k, 0, 0, c, fx, fy) * H)
        if gam[e] != 0.0 and P.p >= 1:
            nu = _lambda(P, m, e, ce) * m.h / (2 * P.p)
            ux = m.poly(ce, 1, 0, c, X, Y)
            uy = m.poly(ce, 0, 1, c, X, Y) if P.dim == 2 else 0 * X
            for k in range(K):
                g = m.basis(k, 1, 0, c, X, Y) * ux
                if P.dim == 2:
                    g = g + m.basis(k, 0, 1, c, X, Y) * uy
                R[k] -= gam[e] * nu * np.sum(W * g)
        for k in range(K):
            i, j = k % m.n1, k // m.n1
            Mkk = (m.h / 2) * 2 / (2 * i + 1)
            if P.dim == 2:
                Mkk *= (m.h / 2) * 2 / (2 * j + 1)
            L[k, e] = R[k] / Mkk
    return L


# ---------------------------------------------------------------------------------
# Euler system (Sec. 5.6), 1D and 2D: U = (rho, rho v, rho E), p = (gamma - 1)(rho E -
# rho |v|^2 / 2)
# ---------------------------------------------------------------------------------
def _euler_Fn(g, q, n):
    """F(U) n for states q of shape (d + 2, npts) and a unit normal n = (nx, ny)."""
    d = q.shape[0] - 2
    rho, en = q[0], q[d + 1]
    v = [q[1 + a] / rho for a in range(d)]
    pr = (g - 1.0) * (en - 0.5 * sum(q[1 + a] * v[a] for a in range(d)))
    vn = sum(v[a] * n[a] for a in range(d))
    out = [rho * vn] + [q[1 + a] * vn + pr * n[a] for a in range(d)] + [(en + pr) * vn]
    return np.array(out)


def _euler_speed(g, q, n=None):
    d = q.shape[0] - 2
    rho, en = q[0], q[d + 1]
    v = [q[1 + a] / rho for a in range(d)]
    pr = (g - 1.0) * (en - 0.5 * sum(q[1 + a] * v[a] for a in range(d)))
    vv = np.abs(sum(v[a] * n[a] for a in range(d))) if n is not None else np.sqrt(sum(x * x for x in v))
    return vv + np.sqrt(g * pr / rho)


def euler_residual(P, U):
    """Euler residual on a 1D or 2D mesh.  The flux integrals use the (p+2)-point Gauss
    rule per direction of the scheme (the flux is not a polynomial, so the rule is part
    of the method); the polynomial integrals of the stabilization use the 24-point rule.
    The sensor is the scalar one applied to the density."""
    import dataclasses
    d = P.dim
    m = Mesh(dataclasses.replace(P, flux="advect"))
    E, g, K = P.E, P.gas_gamma, (P.p + 1) ** d
    nc = d + 2
    Ps = dataclasses.replace(P, flux="advect", bc=tuple("outflow" if b in ("reflect", "state") else b for b in P.bc))
    if P.stab in ("weno", "zhao"):
        gam = sensor(Ps, U[:K])
    else:
        gam = np.full(E, 1.0 if P.stab == "lo" else 0.0)
    gq, wq = npleg.leggauss(P.p + 2)
    L = np.zeros((nc * K, E))
    for e in range(E):
        c = m.centre(e)
        ce = [U[comp * K:(comp + 1) * K, e] for comp in range(nc)]
        state = lambda X, Y, cc=ce, ctr=c: np.array([m.poly(cc[comp], 0, 0, ctr, X, Y) for comp in range(nc)])
        if d == 1:
            X = c[0] + 0.5 * m.h * gq
            Y = 0 * X
            W = 0.5 * m.h * wq
        else:
            X, Y = np.meshgrid(c[0] + 0.5 * m.h * gq, c[1] + 0.5 * m.h * gq, indexing="xy")
            X, Y = X.ravel(), Y.ravel()
            W = np.outer(wq, wq).ravel() * 0.25 * m.h ** 2
        q = state(X, Y)
        Fx = _euler_Fn(g, q, (1.0, 0.0))
        Fy = _euler_Fn(g, q, (0.0, 1.0)) if d == 2 else 0 * Fx
        R = np.zeros((nc, K))
        for k in range(K):
            bx = m.basis(k, 1, 0, c, X, Y)
            by = m.basis(k, 0, 1, c, X, Y) if d == 2 else 0 * X
            R[:, k] = ((Fx * bx + Fy * by) * W).sum(axis=1)
        lam = np.max(_euler_speed(g, q))
        for f in range(2 * d):
            n = [(-1.0, 0.0), (1.0, 0.0), (0.0, -1.0), (0.0, 1.0)][f]
            if d == 1:
                fx, fy, fw = np.array([c[0] + 0.5 * m.h * n[0]]), np.zeros(1), np.ones(1)
            elif f < 2:
                fx, fy, fw = np.full(P.p + 2, c[0] + 0.5 * m.h * n[0]), c[1] + 0.5 * m.h * gq, 0.5 * m.h * wq
            else:
                fx, fy, fw = c[0] + 0.5 * m.h * gq, np.full(P.p + 2, c[1] + 0.5 * m.h * n[1]), 0.5 * m.h * wq
            um = state(fx, fy)
            lam = max(lam, np.max(_euler_speed(g, um)))
            nb, cn = m.nbr(e, f)
            if nb is not None:
                up = np.array([m.poly(U[comp * K:(comp + 1) * K, nb], 0, 0, cn, fx, fy) for comp in range(nc)])
            elif P.bc[f] in ("reflect", "state"):
                up = um.copy()
                mn = sum(um[1 + a] * n[a] for a in range(d))
                wall = np.ones(um.shape[1], dtype=bool)
                if P.bc[f] == "state":
                    # per face point: a prescribed state or a wall, by the point's position
                    # along the side against the moving split
                    along = fy if f < 2 else fx
                    ch = np.where(along < P.bsplit[f] + P.bspeed[f] * P.t, P.bbelow[f], P.babove[f])
                    wall = ch == 2
                    for i in (0, 1):
                        sel = ch == i
                        up[:, sel] = np.asarray(P.bstate[i][:nc], dtype=np.float64)[:, None]
                for a in range(d):
                    up[1 + a] = np.where(wall, um[1 + a] - 2.0 * mn * n[a], up[1 + a])
            else:
                up = um.copy()
            s = np.maximum(_euler_speed(g, um, n), _euler_speed(g, up, n))
            H = 0.5 * (_euler_Fn(g, um, n) + _euler_Fn(g, up, n)) - 0.5 * s * (up - um)
            for k in range(K):
                R[:, k] -= (H * m.basis(k, 0, 0, c, fx, fy) * fw).sum(axis=1)
        if gam[e] != 0.0:
            nu = (P.lambda_nu if P.lambda_nu > 0 else lam) * m.h / (2 * P.p)
            X2, Y2, W2 = m.vol_pts(e)
            for comp in range(nc):
                ux = m.poly(ce[comp], 1, 0, c, X2, Y2)
                uy = m.poly(ce[comp], 0, 1, c, X2, Y2) if d == 2 else 0 * X2
                for k in range(K):
                    gk = m.basis(k, 1, 0, c, X2, Y2) * ux
                    if d == 2:
                        gk = gk + m.basis(k, 0, 1, c, X2, Y2) * uy
                    R[comp, k] -= gam[e] * nu * np.sum(W2 * gk)
        for k in range(K):
            i, j = k % (P.p + 1), k // (P.p + 1)
            Mkk = m.h / (2 * i + 1)
            if d == 2:
                Mkk *= m.h / (2 * j + 1)
            L[k::K, e] = R[:, k] / Mkk
    return L
