"""Constitutive relations of the LGDM (Sec. 2.1 and Appendix A).

All functions accept real or complex numpy arrays; branch decisions (the
damage threshold, the history maximum, the zero-radicand guard) look at the
real part only, so a complex-step perturbation differentiates the selected
branch.
"""
import numpy as np


def damage(kappa, kappa0, alpha, beta):
    """Damage D(kappa) and dD/dkappa, exponential softening (Eq. A.1).

    D = 1 - (kappa0/kappa) * (1 - alpha + alpha * exp(-beta (kappa - kappa0)))
    for kappa > kappa0, and D = 0 (with zero slope) for kappa <= kappa0.
    """
    kappa = np.asarray(kappa)
    on = np.real(kappa) > kappa0
    ks = np.where(on, kappa, 2.0 * kappa0)          # keep the unused branch finite
    ex = np.exp(-beta * (ks - kappa0))
    soft = 1.0 - alpha + alpha * ex
    D = np.where(on, 1.0 - (kappa0 / ks) * soft, 0.0)
    dD = np.where(on, (kappa0 / ks**2) * soft + (kappa0 / ks) * alpha * beta * ex, 0.0)
    return D, dD


def history(kappa_hist, ebar_gp):
    """Trial history kappa = max(kappa_hist, ebar) and the loading flag (Eq. A.2).

    chi = 1 when the micro-equivalent strain exceeds the stored history (the
    history then follows it, d kappa / d ebar = 1), else 0.
    """
    chi = np.real(ebar_gp) > np.real(kappa_hist)
    kappa = np.where(chi, ebar_gp, kappa_hist)
    return kappa, chi.astype(float)


def interaction(D, R, eta):
    """Interaction function g(D) and dg/dD (Eq. A.4); g(0) = 1, g(1) = R."""
    den = 1.0 - np.exp(-eta)
    e = np.exp(-eta * D)
    g = ((1.0 - R) * e + R - np.exp(-eta)) / den
    dg = -eta * (1.0 - R) * e / den
    return g, dg


def lame(E, nu):
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = E / (2.0 * (1.0 + nu))
    return lam, mu


def elasticity_matrix(dim, E, nu):
    """Isotropic elasticity in Voigt form with engineering shear strains.

    1D: [E].  2D: plane strain, order (xx, yy, xy).  3D: order
    (xx, yy, zz, yz, xz, xy).
    """
    if dim == 1:
        return np.array([[E]], dtype=float)
    lam, mu = lame(E, nu)
    if dim == 2:
        return np.array([[lam + 2 * mu, lam, 0.0],
                         [lam, lam + 2 * mu, 0.0],
                         [0.0, 0.0, mu]])
    C = np.zeros((6, 6))
    C[:3, :3] = lam
    C[np.arange(3), np.arange(3)] += 2 * mu
    C[np.arange(3, 6), np.arange(3, 6)] = mu
    return C


def evm_coefficients(nu, k, variant=0):
    """Coefficients (a, b2, cJ) of eps_eq = a I1 + sqrt(b2 I1^2 + cJ J2) / (2k).

    Eq. A.3 with J2 = 1/2 dev(eps):dev(eps).  variant 0 uses cJ = 12k/(1+nu)^2,
    the value for which uniaxial stress gives eps_eq equal to the axial
    strain; variant 1 takes the printed 2k/(1-nu)^2 literally.
    """
    a = (k - 1.0) / (2.0 * k * (1.0 - 2.0 * nu))
    b2 = ((k - 1.0) / (1.0 - 2.0 * nu)) ** 2
    cJ = 12.0 * k / (1.0 + nu) ** 2 if variant == 0 else 2.0 * k / (1.0 - nu) ** 2
    return a, b2, cJ


def equivalent_strain(eps, dim, nu, k, variant=0):
    """Modified von Mises equivalent strain and its gradient (Eq. A.3).

    ``eps`` has Voigt components (engineering shear) in its last axis.  Plane
    strain keeps eps_zz = 0.  In 1D the equivalent strain is the axial strain.
    Where the radicand vanishes the square-root part and its gradient are 0.
    Returns (eps_eq, d eps_eq / d eps) with d in the same Voigt layout.
    """
    eps = np.asarray(eps)
    if dim == 1:
        return eps[..., 0], np.ones_like(eps)
    a, b2, cJ = evm_coefficients(nu, k, variant)
    if dim == 2:
        exx, eyy, gxy = eps[..., 0], eps[..., 1], eps[..., 2]
        I1 = exx + eyy
        ezz = 0.0
        shear2 = gxy**2
        dI1 = np.stack([np.ones_like(exx), np.ones_like(exx), np.zeros_like(exx)], -1)
        dJ2 = np.stack([exx - I1 / 3.0, eyy - I1 / 3.0, gxy / 2.0], -1)
    else:
        exx, eyy, ezz = eps[..., 0], eps[..., 1], eps[..., 2]
        gyz, gxz, gxy = eps[..., 3], eps[..., 4], eps[..., 5]
        I1 = exx + eyy + ezz
        shear2 = gyz**2 + gxz**2 + gxy**2
        one, zero = np.ones_like(exx), np.zeros_like(exx)
        dI1 = np.stack([one, one, one, zero, zero, zero], -1)
        dJ2 = np.stack([exx - I1 / 3.0, eyy - I1 / 3.0, ezz - I1 / 3.0,
                        gyz / 2.0, gxz / 2.0, gxy / 2.0], -1)
    # eps:eps with tensor shear components (eps_ij = gamma_ij / 2)
    epseps = exx**2 + eyy**2 + ezz**2 + 0.5 * shear2
    J2 = 0.5 * (epseps - I1**2 / 3.0)
    Q = b2 * I1**2 + cJ * J2
    live = np.real(Q) > 0.0
    root = np.sqrt(np.where(live, Q, 1.0))
    eq = a * I1 + np.where(live, root, 0.0) / (2.0 * k)
    dQ = 2.0 * b2 * I1[..., None] * dI1 + cJ * dJ2
    droot = np.where(live[..., None], dQ / (2.0 * root[..., None]), 0.0)
    d = a * dI1 + droot / (2.0 * k)
    return eq, d


def equivalent_strain_hessian(eps, dim, nu, k, variant=0):
    """Second derivative of the equivalent strain (Eq. A.3) with respect to the
    Voigt strain (engineering shear), shape (..., nv, nv).

    With Q = b2 I1^2 + cJ J2 and eps_eq = a I1 + sqrt(Q) / (2k):
    d2 eps_eq = [d2Q / (2 sqrt Q) - dQ (x) dQ / (4 Q^(3/2))] / (2k), where
    dQ = 2 b2 I1 dI1 + cJ dJ2 and d2Q = 2 b2 dI1 (x) dI1 + cJ d2J2; d2J2 is
    delta_ij - 1/3 between normal components and 1/2 on each shear component
    (J2 = 1/2 dev(eps):dev(eps), tensor shear gamma/2).  Zero where Q vanishes
    and in 1D (eps_eq is the axial strain there).
    """
    eps = np.asarray(eps)
    nv = eps.shape[-1]
    if dim == 1:
        return np.zeros(eps.shape + (1,), dtype=eps.dtype)
    a, b2, cJ = evm_coefficients(nu, k, variant)
    nn = dim                                             # normal components (plane strain: xx, yy)
    I1 = np.sum(eps[..., :nn], axis=-1)
    dI1 = np.zeros(nv)
    dI1[:nn] = 1.0
    dJ2 = np.concatenate([eps[..., :nn] - I1[..., None] / 3.0, eps[..., nn:] / 2.0], axis=-1)
    ee = np.sum(eps[..., :nn] ** 2, axis=-1) + 0.5 * np.sum(eps[..., nn:] ** 2, axis=-1)
    J2 = 0.5 * (ee - I1 ** 2 / 3.0)
    Q = b2 * I1 ** 2 + cJ * J2
    d2J2 = np.zeros((nv, nv))
    d2J2[:nn, :nn] = np.eye(nn) - 1.0 / 3.0
    d2J2[nn:, nn:] = 0.5 * np.eye(nv - nn)
    dQ = 2.0 * b2 * I1[..., None] * dI1 + cJ * dJ2
    d2Q = 2.0 * b2 * np.outer(dI1, dI1) + cJ * d2J2
    live = np.real(Q) > 0.0
    Qs = np.where(live, Q, 1.0)
    root = np.sqrt(Qs)
    H = (d2Q / (2.0 * root[..., None, None])
         - np.einsum("...i,...j->...ij", dQ, dQ) / (4.0 * (Qs * root)[..., None, None])) / (2.0 * k)
    return np.where(live[..., None, None], H, 0.0)


def free_energy_density(D, eps, C_eps, h, eps_eq, ebar, g, c, grad_ebar):
    """Free energy density (Eq. 1).

    1/2 (1-D) eps:C:eps + 1/2 h (eps_eq - ebar)^2 + 1/2 g h c grad(ebar).grad(ebar).
    ``C_eps`` is C:eps in Voigt form, so eps:C:eps = sum(eps * C_eps).
    """
    return (0.5 * (1.0 - D) * np.sum(eps * C_eps, axis=-1)
            + 0.5 * h * (eps_eq - ebar) ** 2
            + 0.5 * g * h * c * np.sum(grad_ebar * grad_ebar, axis=-1))
