"""Moebius domain-wall operator, FP64, plain numpy (oracle; test infrastructure only).

The paper (Sec. "Current State of the Art") states the problem: a Dirac matrix on
L^3 x T x L5 x Nc x Ns that is a radius-one stencil with small dense 12x12 diagonal
blocks, solved with CG on the normal equations and red-black preconditioning, for the
Moebius domain-wall discretisation.  It prints no formula; the readings used here:

  Wilson hop    (H psi)(x) = sum_mu (1 - gamma_mu) U_mu(x) psi(x+mu)
                           + (1 + gamma_mu) U_mu(x-mu)^dagger psi(x-mu)
                periodic in space; the t-links crossing T-1 -> 0 carry t_bc (= -1,
                antiperiodic), folded into the links by ``boundary_links``.
  Wilson op     D_W = (4 - M5) - H/2                 (domain-wall height M5)
  s-shift       (B psi)_s = P_- psi_{s+1} + P_+ psi_{s-1},
                with psi_{Ls} -> -m_f psi_0 and psi_{-1} -> -m_f psi_{Ls-1}
  Moebius 5D    D = D_W (b5 + c5 B) + (1 - B)
                i.e. (D psi)_s = (b5 D_W + 1) psi_s + (c5 D_W - 1)(B psi)_s
  even-odd      D5 = b5 + c5 B,  A5 = (4 - M5) D5 + (1 - B) = alpha + beta B,
                alpha = (4-M5) b5 + 1, beta = (4-M5) c5 - 1
                D = [[A5, -H_eo D5 / 2], [-H_oe D5 / 2, A5]]   (parity = x+y+z+t mod 2)
                M_pc = 1 - (1/4) A5^-1 H_oe D5 A5^-1 H_eo D5   on odd sites
                b~_o = A5^-1 (b_o + H_oe D5 A5^-1 b_e / 2)
                x_e  = A5^-1 (b_e + H_eo D5 x_o / 2)
Field layouts are those of ``inputs``: 4D [..., t, z, y, x, spin, colour],
5D [..., s, t, z, y, x, spin, colour], links [t, z, y, x, mu, a, b].
"""
from dataclasses import dataclass
import numpy as np

from .gamma import GAMMA, GAMMA5, ID4

SPIN_AXIS = -2
MU_AXIS = {0: -3, 1: -4, 2: -5, 3: -6}  # x, y, z, t axis of a [.., t,z,y,x,4,3] field
S_AXIS = -7


@dataclass
class MobiusParams:
    Ls: int
    b5: float = 1.5
    c5: float = 0.5
    M5: float = 1.3
    mf: float = 0.05
    t_bc: float = -1.0

    @property
    def alpha(self):
        return (4.0 - self.M5) * self.b5 + 1.0

    @property
    def beta(self):
        return (4.0 - self.M5) * self.c5 - 1.0


# ---------------------------------------------------------------- 4D pieces
def boundary_links(U, t_bc=-1.0):
    """Links with the time boundary phase folded into U_t(x) at t = T-1."""
    Ub = np.array(U, dtype=np.complex128, copy=True)
    Ub[-1, :, :, :, 3] *= t_bc
    return Ub


def shift(f, mu, sign):
    """f(x + sign*mu_hat) for a field whose trailing axes are [t,z,y,x,4,3]."""
    return np.roll(f, -sign, axis=MU_AXIS[mu])


def _link_shift(Umu, mu, sign):
    """U_mu(x + sign*mu_hat) for a link array [t,z,y,x,3,3]."""
    return np.roll(Umu, -sign, axis={0: 3, 1: 2, 2: 1, 3: 0}[mu])


def hop(Ub, psi, dagger=False):
    """Wilson hop H psi (or H^dagger psi = gamma5 H gamma5 psi) with links Ub
    that already carry the boundary phase."""
    sig = -1.0 if dagger else 1.0
    out = np.zeros_like(psi, dtype=np.complex128)
    for mu in range(4):
        Umu = Ub[:, :, :, :, mu]
        fwd = shift(psi, mu, +1) @ np.swapaxes(Umu, -1, -2)          # U_mu(x) psi(x+mu)
        bwd = shift(psi, mu, -1) @ np.conj(_link_shift(Umu, mu, -1))  # U_mu(x-mu)^+ psi(x-mu)
        out += (ID4 - sig * GAMMA[mu]) @ fwd + (ID4 + sig * GAMMA[mu]) @ bwd
    return out


def wilson(Ub, psi, M5, dagger=False):
    """D_W psi = (4 - M5) psi - H psi / 2 (D_W^dagger with dagger=True)."""
    return (4.0 - M5) * psi - 0.5 * hop(Ub, psi, dagger)


def gamma5(psi):
    return GAMMA5 @ psi


# ---------------------------------------------------------------- s-direction pieces
def b_matrices(Ls, mf):
    """Ls x Ls matrices of B on the P_- (upper-spin) and P_+ (lower-spin) parts."""
    Bm = np.zeros((Ls, Ls))
    Bp = np.zeros((Ls, Ls))
    for s in range(Ls - 1):
        Bm[s, s + 1] = 1.0
        Bp[s + 1, s] = 1.0
    Bm[Ls - 1, 0] = -mf
    Bp[0, Ls - 1] = -mf
    return Bm, Bp


def s_apply(Mm, Mp, psi):
    """out_s = sum_s' M[s, s'] psi_s' with Mm on spins 0,1 (P_-) and Mp on 2,3 (P_+)."""
    ps = np.moveaxis(psi, S_AXIS, -1)  # [..., t,z,y,x,4,3,Ls]
    up = ps[..., 0:2, :, :] @ np.asarray(Mm).T
    dn = ps[..., 2:4, :, :] @ np.asarray(Mp).T
    return np.moveaxis(np.concatenate([up, dn], axis=-3), -1, S_AXIS)


def s_matrices(p, which, dagger=False, mf=None):
    """(Mm, Mp) of one s-operator: 'B', 'D5', 'A5', 'A5inv', 'D5inv'.  The inverses are
    plain dense inverses of the matrices built from the definition."""
    mf = p.mf if mf is None else mf
    Bm, Bp = b_matrices(p.Ls, mf)
    I = np.eye(p.Ls)
    if which == "B":
        mats = (Bm, Bp)
    elif which == "D5":
        mats = (p.b5 * I + p.c5 * Bm, p.b5 * I + p.c5 * Bp)
    elif which == "A5":
        mats = (p.alpha * I + p.beta * Bm, p.alpha * I + p.beta * Bp)
    elif which == "A5inv":
        mats = (np.linalg.inv(p.alpha * I + p.beta * Bm),
                np.linalg.inv(p.alpha * I + p.beta * Bp))
    elif which == "D5inv":
        mats = (np.linalg.inv(p.b5 * I + p.c5 * Bm),
                np.linalg.inv(p.b5 * I + p.c5 * Bp))
    else:
        raise ValueError(which)
    if dagger:  # real matrices: adjoint = transpose
        mats = (mats[0].T, mats[1].T)
    return mats


def s_op(p, which, psi, dagger=False, mf=None):
    Mm, Mp = s_matrices(p, which, dagger, mf)
    return s_apply(Mm, Mp, psi)


# ---------------------------------------------------------------- 5D operator
def mobius(Ub, psi, p, mf=None, dagger=False):
    """Full 5D Moebius operator D psi (or D^dagger psi); mf overrides the quark mass
    (mf=1 gives the Pauli-Villars operator used for source injection)."""
    if not dagger:
        Bpsi = s_op(p, "B", psi, mf=mf)
        return wilson(Ub, p.b5 * psi + p.c5 * Bpsi, p.M5) + psi - Bpsi
    # D^dagger = D5^dagger D_W^dagger + 1 - B^dagger
    w = wilson(Ub, psi, p.M5, dagger=True)
    return (p.b5 * w + p.c5 * s_op(p, "B", w, dagger=True, mf=mf)
            + psi - s_op(p, "B", psi, dagger=True, mf=mf))


# ---------------------------------------------------------------- even-odd
def parity_mask(dims):
    X, Y, Z, T = dims
    t, z, y, x = np.meshgrid(np.arange(T), np.arange(Z), np.arange(Y), np.arange(X),
                             indexing="ij")
    return (x + y + z + t) % 2  # [t,z,y,x]


def on_parity(psi, par, parity):
    """psi restricted to sites of the given parity (zero elsewhere)."""
    m = (par == parity)[..., None, None]
    return np.where(m, psi, 0.0)


def mpc(Ub, psi_o, p):
    """M_pc psi_o = psi_o - (1/4) A5^-1 H_oe D5 A5^-1 H_eo D5 psi_o (psi_o odd-supported)."""
    t = s_op(p, "A5inv", hop(Ub, s_op(p, "D5", psi_o)))
    u = s_op(p, "A5inv", hop(Ub, s_op(p, "D5", t)))
    return psi_o - 0.25 * u


def mpc_dag(Ub, psi_o, p):
    """M_pc^dagger = 1 - (1/4) D5^+ H_eo^+ A5^-+ D5^+ H_oe^+ A5^-+ (H^+ = gamma5 H gamma5)."""
    t = s_op(p, "D5", hop(Ub, s_op(p, "A5inv", psi_o, dagger=True), dagger=True), dagger=True)
    u = s_op(p, "D5", hop(Ub, s_op(p, "A5inv", t, dagger=True), dagger=True), dagger=True)
    return psi_o - 0.25 * u


def mpc_sym(Ub, psi_o, p):
    """Symmetric even-odd form.  D D5^-1 = [[A~, -H_eo/2], [-H_oe/2, A~]] with the
    s-local diagonal block A~ = A5 D5^-1; its odd-site Schur complement with both
    diagonal inverses on the left of their hops is
        M_sym = 1 - (1/4) A~^-1 H_oe A~^-1 H_eo,   A~^-1 = D5 A5^-1
    (= D5 M_pc D5^-1).  The odd system M_sym y = D5 b~_o gives x_o = D5^-1 y."""
    t = s_op(p, "D5", s_op(p, "A5inv", hop(Ub, psi_o)))
    u = s_op(p, "D5", s_op(p, "A5inv", hop(Ub, t)))
    return psi_o - 0.25 * u


def mpc_sym_dag(Ub, psi_o, p):
    """M_sym^dagger = 1 - (1/4) (H^+)_oe A~^-+ (H^+)_eo A~^-+,  A~^-+ = A5^-+ D5^+."""
    xd = lambda f: s_op(p, "A5inv", s_op(p, "D5", f, dagger=True), dagger=True)
    t = hop(Ub, xd(psi_o), dagger=True)
    u = hop(Ub, xd(t), dagger=True)
    return psi_o - 0.25 * u


def prepare_source(Ub, b, p, par):
    """b~_o = A5^-1 (b_o + (1/2) H_oe D5 A5^-1 b_e)."""
    be = on_parity(b, par, 0)
    bo = on_parity(b, par, 1)
    return s_op(p, "A5inv", bo + 0.5 * hop(Ub, s_op(p, "D5", s_op(p, "A5inv", be))))


def reconstruct(Ub, b, x_o, p, par):
    """Full solution from the odd part: x_e = A5^-1 (b_e + (1/2) H_eo D5 x_o)."""
    be = on_parity(b, par, 0)
    xe = s_op(p, "A5inv", be + 0.5 * hop(Ub, s_op(p, "D5", x_o)))
    return xe + x_o


def hop_eo(Ub, psi, par, out_parity, dagger=False):
    """H restricted to out_parity <- 1-out_parity (the half-lattice hop)."""
    return on_parity(hop(Ub, on_parity(psi, par, 1 - out_parity), dagger), par, out_parity)
