"""Independent numpy restatement of one time step in MOMENT space.

Test helper only.  The FP64 oracle in ``oracle/`` works in velocity space with
explicit M and M^-1 products (Eq. 10, 11, 14, 15, 25-29); this module instead
uses the moment-space closed forms the paper gives for the implementation
(Eq. 21-23 for the phase field, Eq. 36-37 for the hydrodynamics), the
closed-form inverse M^-1 = M^T diag(1/9, 1/36, 1/36, 1/6, 1/12, 1/6, 1/12, 1/4, 1/4),
a padded-array ghost construction and a vectorised push streaming.  Agreement
of the two to round-off pins both.
"""
import numpy as np

CZ = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
CR = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
M = np.array([
    [1, 1, 1, 1, 1, 1, 1, 1, 1],
    [-4, -1, -1, -1, -1, 2, 2, 2, 2],
    [4, -2, -2, -2, -2, 1, 1, 1, 1],
    [0, 1, 0, -1, 0, 1, -1, -1, 1],
    [0, -2, 0, 2, 0, 1, -1, -1, 1],
    [0, 0, 1, 0, -1, 1, 1, -1, -1],
    [0, 0, -2, 0, 2, 1, 1, -1, -1],
    [0, 1, -1, 1, -1, 0, 0, 0, 0],
    [0, 0, 0, 0, 0, 1, -1, 1, -1]], dtype=np.float64)
MINV = M.T @ np.diag([1 / 9, 1 / 36, 1 / 36, 1 / 6, 1 / 12, 1 / 6, 1 / 12, 1 / 4, 1 / 4])
OPP = np.array([0, 3, 4, 1, 2, 7, 8, 5, 6])
RMIR = np.array([0, 1, 4, 3, 2, 8, 7, 6, 5])


def padded(field, zper):
    """[nz][nr] -> [nz+4][nr+4] with the axis/wall mirror and periodic ghosts."""
    nz, nr = field.shape
    out = np.zeros((nz + 4, nr + 4))
    out[2:-2, 2:-2] = field
    # r direction: axis mirror (j=-1 <- 0, j=-2 <- 1), wall mirror (nr <- nr-1, nr+1 <- nr-2)
    out[2:-2, 1] = field[:, 0]
    out[2:-2, 0] = field[:, 1]
    out[2:-2, nr + 2] = field[:, nr - 1]
    out[2:-2, nr + 3] = field[:, nr - 2]
    if zper:
        out[0:2, :] = out[nz:nz + 2, :]
        out[nz + 2:nz + 4, :] = out[2:4, :]
    else:
        out[1, :] = out[2, :]
        out[0, :] = out[3, :]
        out[nz + 2, :] = out[nz + 1, :]
        out[nz + 3, :] = out[nz, :]
    return out


def stencils(phi, zper):
    nz, nr = phi.shape
    P = padded(phi, zper)

    def sh(a, b):
        return P[2 + a:2 + a + nz, 2 + b:2 + b + nr]

    gz = np.zeros_like(phi)
    gr = np.zeros_like(phi)
    lap = np.zeros_like(phi)
    for i in range(1, 9):
        x1 = sh(CZ[i], CR[i])
        x2 = sh(2 * CZ[i], 2 * CR[i])
        gz += W[i] * CZ[i] * (8 * x1 - x2) / 2.0
        gr += W[i] * CR[i] * (8 * x1 - x2) / 2.0
        lap += W[i] * (16 * x1 - x2 - 15 * phi) / 2.0
    return gz, gr, lap


def step(case, f, g, chi_z, chi_r, p_prev):
    nz, nr = f.shape[1:]
    zper = bool(case.get("z_periodic", 0))
    r = (np.arange(nr) + 0.5)[None, :] * np.ones((nz, 1))
    phi = f.sum(axis=0) / r
    gz, gr, lap = stencils(phi, zper)
    rl, rg = case["rho_l"], case["rho_g"]
    rho = phi * rl + (1 - phi) * rg
    nu = phi * case["nu_l"] + (1 - phi) * case["nu_g"]
    sig, Wd, mob = case["sigma"], case["W"], case["mobility"]
    beta, kap = 12 * sig / Wd, 1.5 * sig * Wd
    mu = 4 * beta * phi * (phi - 1) * (phi - 0.5) - kap * lap
    mut = mu - kap * gr / r
    Fsz, Fsr = mut * gz, mut * gr
    Gz = (rho - rl) * case.get("grav_z", 0.0)
    Gr = np.zeros_like(phi)
    gn = np.sqrt(gz ** 2 + gr ** 2)
    nz_, nr_ = gz / (gn + case["n_eps"]), gr / (gn + case["n_eps"])
    lam = 4 * phi * (1 - phi) / Wd
    tau_f = 3 * mob + 0.5
    tau_g = 3 * nu + 0.5
    sf = [np.full_like(phi, 1 / tau_f) if s < 0 else np.full_like(phi, s) for s in case["sf"]]
    sg = [1 / tau_g if s < 0 else np.full_like(phi, s) for s in case["sg"]]
    mg = np.einsum("ab,bzr->azr", M, g)
    Jz, Jr, S0 = mg[3], mg[5], mg[0] - g[0]
    dzrho, drrho = (rl - rg) * gz, (rl - rg) * gr
    sp = (sg[1] + sg[2] - sg[1] * sg[2]) / (2 * sg[1] * sg[2])
    uz = (Jz + 0.5 * r * (Fsz + Gz)) / (r * rho)
    Dr = r * rho + nu * rho / r
    if case.get("p_coupling", 0) == 1:
        ps = p_prev
        ur = (Jr + 0.5 * (r * (Fsr + Gr) + ps)) / Dr
        p = 0.6 * (S0 / r + 0.5 * (uz * dzrho + ur * drrho)
                   - (2 / 3) * rho * (uz ** 2 + ur ** 2) - sp * (4 / 9) * rho * ur / r)
    else:
        a = (Jr + 0.5 * r * (Fsr + Gr)) / Dr
        b = 0.5 / Dr
        A0 = 0.6 * (S0 / r + 0.5 * uz * dzrho - (2 / 3) * rho * uz ** 2)
        A1 = 0.6 * (0.5 * drrho - sp * (4 / 9) * rho / r)
        A2 = 0.6 * (2 / 3) * rho
        qa, qb, qc = A2 * b * b, 1 - A1 * b + 2 * A2 * a * b, -(A0 + A1 * a - A2 * a * a)
        p = -2 * qc / (qb + np.sqrt(qb * qb - 4 * qa * qc))
        ps = p
        ur = a + b * p
    Fz = r * (Fsz + Gz)
    Fr = r * (Fsr + Gr) + ps - 2 * rho * nu * ur / r
    # ---- phase field, Eq. 19 in moment space with Eq. 21-23
    cz_new = r * phi * uz
    cr_new = r * phi * ur + mob * phi
    mR1 = (cz_new - chi_z) + r * nz_ * lam / 3
    mR2 = (cr_new - chi_r) + r * nr_ * lam / 3
    mf = np.einsum("ab,bzr->azr", M, f)
    rp = r * phi
    meq = np.stack([rp, -2 * rp, rp, cz_new, -cz_new, cr_new, -cr_new, 0 * rp, 0 * rp])
    mR = np.stack([0 * rp, 0 * rp, 0 * rp, mR1, -mR1, mR2, -mR2, 0 * rp, 0 * rp])
    mfp = np.stack([mf[k] - sf[k] * (mf[k] - meq[k]) + (1 - sf[k] / 2) * mR[k] for k in range(9)])
    fpost = np.einsum("ab,bzr->azr", MINV, mfp)
    # ---- hydrodynamics, Eq. 24 in moment space with Eq. 36-37
    u2 = uz ** 2 + ur ** 2
    geq = r * np.stack([0 * rp, 3 * (2 * p + rho * u2), -3 * (3 * p + rho * u2), rho * uz, -rho * uz,
                        rho * ur, -rho * ur, rho * (uz ** 2 - ur ** 2), rho * ur * uz])
    dz_rr, dr_rr = r * dzrho, rho + r * drrho
    udr = uz * dz_rr + ur * dr_rr
    MT = np.stack([r * (uz * dzrho + ur * drrho), 2 * rho * ur, -udr - rho * ur, Fz, -Fz, Fr, -Fr,
                   (2 / 3) * (uz * dz_rr - ur * dr_rr), (1 / 3) * (uz * dr_rr + ur * dz_rr)])
    mgp = np.stack([mg[k] - sg[k] * (mg[k] - geq[k]) + (1 - sg[k] / 2) * MT[k] for k in range(9)])
    gpost = np.einsum("ab,bzr->azr", MINV, mgp)
    # ---- streaming (push) with the boundary rules
    fn, gnew = np.zeros_like(f), np.zeros_like(g)
    K, J = np.meshgrid(np.arange(nz), np.arange(nr), indexing="ij")
    for i in range(9):
        kt, jt = K + CZ[i], J + CR[i]
        if zper:
            kt = kt % nz
            zout = np.zeros_like(kt, dtype=bool)
        else:
            zout = (kt < 0) | (kt >= nz)
        wall = zout | (jt >= nr)
        axis = (~wall) & (jt < 0)
        inner = ~(wall | axis)
        fn[OPP[i], K[wall], J[wall]] = fpost[i][wall]
        gnew[OPP[i], K[wall], J[wall]] = gpost[i][wall]
        fn[RMIR[i], kt[axis], 0] = fpost[i][axis]
        gnew[RMIR[i], kt[axis], 0] = gpost[i][axis]
        fn[i, kt[inner], jt[inner]] = fpost[i][inner]
        gnew[i, kt[inner], jt[inner]] = gpost[i][inner]
    fields = dict(phi=phi, rho=rho, uz=uz, ur=ur, p=p)
    return fn, gnew, cz_new, cr_new, p, fields
