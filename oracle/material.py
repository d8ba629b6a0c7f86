"""Constitutive law (oracle, FP64).

Sec. III-B: Lame parameters from (E, nu) by Eq. 1; stable Neo-Hookean
material; first Piola-Kirchhoff stress P (Eq. 2); Cauchy stress
sigma = J^-1 P F^T (Eq. 3) and its closed form (Eq. 4).

Reading of the paper (Eq. 2/Eq. 4 as printed give P(I) = mu*I and
sigma(I) = mu*I, i.e. a stressed rest state, and are not the cited
stable Neo-Hookean of Smith et al. 2018): we use the stable Neo-Hookean energy
without the log term,

    Psi(F) = mu/2 (tr F^T F - 3) + lam_hat/2 (J - alpha)^2 - mu^2/(2 lam_hat),
    lam_hat = lam + mu,   alpha = 1 + mu / lam_hat,

whose stress is P = mu F + lam_hat (J - alpha) cof F and whose Cauchy stress is
Eq. 4 with lam -> lam_hat and 1 -> alpha:

    sigma = (mu / J) b + lam_hat (J - alpha) I,   b = F F^T.

It vanishes at rest and linearises to 2 mu eps + lam tr(eps) I, i.e. the
(E, nu) of Eq. 1 exactly.  ``sigma_paper_literal`` evaluates Eq. 4 as printed.

The full stable Neo-Hookean of Smith et al. 2018 (the law Sec. III-B cites,
with its log term) is the second material law, selected per scene:

    Psi(F) = mu_s/2 (I_C - 3) + lam_s/2 (J - alpha_s)^2 - mu_s/2 log(I_C + 1) - Psi(I),
    I_C = tr F^T F,  alpha_s = 1 + 3 mu_s / (4 lam_s),

with mu_s = 4/3 mu and lam_s = lam + 5/6 mu from Eq. 1's (mu, lam), so that it
too is stress-free at rest and linearises to 2 mu eps + lam tr(eps) I.  Its
stress is P = mu_s (1 - 1/(I_C + 1)) F + lam_s (J - alpha_s) cof F and its
Cauchy stress sigma = (mu_s/J)(1 - 1/(I_C + 1)) b + lam_s (J - alpha_s) I.

Vectorisation convention for 9x9 tangents: vec(F)[3*i + j] = F[i, j].
"""
import numpy as np

# Levi-Civita symbol
EPS = np.zeros((3, 3, 3))
for (i, j, k), s in {(0, 1, 2): 1, (1, 2, 0): 1, (2, 0, 1): 1,
                     (0, 2, 1): -1, (2, 1, 0): -1, (1, 0, 2): -1}.items():
    EPS[i, j, k] = s


def lame(E, nu):
    """Eq. 1: mu = E / (2(1+nu)), lam = E nu / ((1+nu)(1-2nu))."""
    mu = E / (2.0 * (1.0 + nu))
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    return mu, lam


def snh_params(E, nu):
    """(mu, lam_hat, alpha) of the rest-stable energy (reading above)."""
    mu, lam = lame(E, nu)
    lam_hat = lam + mu
    return mu, lam_hat, 1.0 + mu / lam_hat


def cofactor(F):
    """cof F = det(F) F^-T, written with the Levi-Civita symbol so that it
    is defined for singular F: cof_ij = 1/2 eps_imn eps_jpq F_mp F_nq."""
    return 0.5 * np.einsum("imn,jpq,...mp,...nq->...ij", EPS, EPS, F, F)


def energy_density(F, mu, lam_hat, alpha):
    """Psi(F), zero at F = I."""
    J = np.linalg.det(F)
    Ic = np.einsum("...ij,...ij->...", F, F)
    return 0.5 * mu * (Ic - 3.0) + 0.5 * lam_hat * (J - alpha) ** 2 - 0.5 * mu * mu / lam_hat


def pk1(F, mu, lam_hat, alpha):
    """P = dPsi/dF = mu F + lam_hat (J - alpha) cof F."""
    J = np.linalg.det(F)
    mu, lam_hat, alpha = (np.asarray(a, dtype=np.float64) for a in (mu, lam_hat, alpha))
    return mu[..., None, None] * F + (lam_hat * (J - alpha))[..., None, None] * cofactor(F)


def dpk1_dF(F, mu, lam_hat, alpha):
    """9x9 tangent dP/dF = mu I + lam_hat vec(cof F) vec(cof F)^T
    + lam_hat (J - alpha) d^2J/dF^2, with d^2J/dF_ij dF_kl = eps_ikm eps_jln F_mn."""
    F = np.asarray(F)
    J = np.linalg.det(F)
    C = cofactor(F).reshape(F.shape[:-2] + (9,))
    HJ = np.einsum("ikm,jln,...mn->...ijkl", EPS, EPS, F).reshape(F.shape[:-2] + (9, 9))
    eye = np.eye(9)
    mu, lam_hat, alpha = (np.asarray(a, dtype=np.float64) for a in (mu, lam_hat, alpha))
    return (mu[..., None, None] * eye + lam_hat[..., None, None] * C[..., :, None] * C[..., None, :]
            + (lam_hat * (J - alpha))[..., None, None] * HJ)


def project_psd(H):
    """Symmetric eigendecomposition, negative eigenvalues clamped to zero."""
    w, Q = np.linalg.eigh(0.5 * (H + np.swapaxes(H, -1, -2)))
    return np.einsum("...ik,...k,...jk->...ij", Q, np.maximum(w, 0.0), Q)


def cauchy_from_pk1(F, P):
    """Eq. 3: sigma = J^-1 P F^T."""
    J = np.linalg.det(F)
    return np.einsum("...ik,...jk->...ij", P, F) / J[..., None, None]


def cauchy(F, mu, lam_hat, alpha):
    """Eq. 4 (rest-stable reading): sigma = (mu/J) F F^T + lam_hat (J - alpha) I."""
    J = np.linalg.det(F)
    b = np.einsum("...ik,...jk->...ij", F, F)
    return (mu / J)[..., None, None] * b + (lam_hat * (J - alpha))[..., None, None] * np.eye(3)


def sigma_paper_literal(F, mu, lam):
    """Eq. 4 exactly as printed: (mu/J) b + lam (J - 1) I (reporting only)."""
    J = np.linalg.det(F)
    b = np.einsum("...ik,...jk->...ij", F, F)
    return (mu / J)[..., None, None] * b + (lam * (J - 1.0))[..., None, None] * np.eye(3)


def sym6(S):
    """3x3 symmetric -> (xx, yy, zz, xy, yz, zx), the storage order of the
    six independent components (Sec. III-C lists nine, six independent)."""
    return np.stack([S[..., 0, 0], S[..., 1, 1], S[..., 2, 2],
                     S[..., 0, 1], S[..., 1, 2], S[..., 2, 0]], axis=-1)


def full33(s6):
    s6 = np.asarray(s6)
    S = np.empty(s6.shape[:-1] + (3, 3))
    S[..., 0, 0], S[..., 1, 1], S[..., 2, 2] = s6[..., 0], s6[..., 1], s6[..., 2]
    S[..., 0, 1] = S[..., 1, 0] = s6[..., 3]
    S[..., 1, 2] = S[..., 2, 1] = s6[..., 4]
    S[..., 2, 0] = S[..., 0, 2] = s6[..., 5]
    return S


# ------------------------------------------------ full stable Neo-Hookean
def snh_log_params(E, nu):
    """(mu_s, lam_s, alpha_s) of the full stable Neo-Hookean (log term):
    Eq. 1's Lame pair mapped by mu_s = 4/3 mu, lam_s = lam + 5/6 mu (the
    small-strain limit is then linear elasticity with E, nu), and the rest
    offset alpha_s = 1 + 3 mu_s / (4 lam_s) that makes P(I) vanish."""
    mu, lam = lame(E, nu)
    mu_s = 4.0 / 3.0 * mu
    lam_s = lam + 5.0 / 6.0 * mu
    return mu_s, lam_s, 1.0 + 0.75 * mu_s / lam_s


def energy_density_log(F, mu_s, lam_s, alpha_s):
    """Psi(F) of the full stable Neo-Hookean, zero at F = I; finite for every
    F (I_C + 1 >= 1), including inverted and collapsed elements."""
    J = np.linalg.det(F)
    Ic = np.einsum("...ij,...ij->...", F, F)
    rest = 0.5 * lam_s * (1.0 - alpha_s) ** 2 - 0.5 * mu_s * np.log(4.0)
    return (0.5 * mu_s * (Ic - 3.0) + 0.5 * lam_s * (J - alpha_s) ** 2
            - 0.5 * mu_s * np.log(Ic + 1.0) - rest)


def pk1_log(F, mu_s, lam_s, alpha_s):
    """P = dPsi/dF = mu_s (1 - 1/(I_C + 1)) F + lam_s (J - alpha_s) cof F."""
    J = np.linalg.det(F)
    Ic = np.einsum("...ij,...ij->...", F, F)
    mu_s, lam_s, alpha_s = (np.asarray(a, dtype=np.float64) for a in (mu_s, lam_s, alpha_s))
    return ((mu_s * (1.0 - 1.0 / (Ic + 1.0)))[..., None, None] * F
            + (lam_s * (J - alpha_s))[..., None, None] * cofactor(F))


def dpk1_dF_log(F, mu_s, lam_s, alpha_s):
    """9x9 tangent: mu_s (1 - 1/(I_C + 1)) I + 2 mu_s/(I_C + 1)^2 vec(F) vec(F)^T
    + lam_s vec(cof F) vec(cof F)^T + lam_s (J - alpha_s) d^2J/dF^2."""
    F = np.asarray(F)
    J = np.linalg.det(F)
    Ic = np.einsum("...ij,...ij->...", F, F)
    f = F.reshape(F.shape[:-2] + (9,))
    C = cofactor(F).reshape(F.shape[:-2] + (9,))
    HJ = np.einsum("ikm,jln,...mn->...ijkl", EPS, EPS, F).reshape(F.shape[:-2] + (9, 9))
    mu_s, lam_s, alpha_s = (np.asarray(a, dtype=np.float64) for a in (mu_s, lam_s, alpha_s))
    a = mu_s * (1.0 - 1.0 / (Ic + 1.0))
    c = 2.0 * mu_s / (Ic + 1.0) ** 2
    return (a[..., None, None] * np.eye(9) + c[..., None, None] * f[..., :, None] * f[..., None, :]
            + lam_s[..., None, None] * C[..., :, None] * C[..., None, :]
            + (lam_s * (J - alpha_s))[..., None, None] * HJ)


def cauchy_log(F, mu_s, lam_s, alpha_s):
    """sigma = J^-1 P F^T = (mu_s/J)(1 - 1/(I_C + 1)) b + lam_s (J - alpha_s) I."""
    J = np.linalg.det(F)
    Ic = np.einsum("...ij,...ij->...", F, F)
    b = np.einsum("...ik,...jk->...ij", F, F)
    return ((mu_s * (1.0 - 1.0 / (Ic + 1.0)) / J)[..., None, None] * b
            + (lam_s * (J - alpha_s))[..., None, None] * np.eye(3))


# material laws by name: (parameters from (E, nu), Psi, P, dP/dF, sigma)
LAWS = {
    "snh": (snh_params, energy_density, pk1, dpk1_dF, cauchy),
    "snh_log": (snh_log_params, energy_density_log, pk1_log, dpk1_dF_log, cauchy_log),
}


def law_params(law, E, nu):
    """The three parameters the law's functions take (the rest-stable law:
    (mu, lam_hat, alpha); the full stable Neo-Hookean: (mu_s, lam_s, alpha_s))."""
    if law == "snh":
        mu, _ = lame(E, nu)
        _, lam_hat, alpha = snh_params(E, nu)
        return mu, lam_hat, alpha
    return snh_log_params(E, nu)
