"""Point-source propagators, the Feynman-Hellmann sequential source and the nucleon
two-point contraction (oracle; test infrastructure only).

Readings (the paper names these pieces but prints no formula; Sec. "Current State of
the Art", Sec. "Performance Measurement Method"):

  injection   5D source eta = D(m_f = 1) P (b at s = 0), (P psi)_s = P_- psi_s + P_+ psi_{s+1}
              (s+1 taken cyclically), so eta's non-zero input slices are s=0 (P_- b)
              and s=Ls-1 (P_+ b) before the Pauli-Villars operator D(1) is applied.
  projection  q = P_- y_0 + P_+ y_{Ls-1} = [P^-1 y]_0, so that q = D_eff^-1 b with
              D_eff^-1 = [P^-1 D(m)^-1 D(1) P]_00 (the overlap operator's inverse).
  FH source   the sequential source is Gamma S(z) at every site z of every timeslice,
              Gamma = gamma_3 gamma_5 acting on the sink spin; solving again gives
              S_FH = D_eff^-1 (sum_z Gamma) S, "all temporal distances for the cost
              of one" (Sec. "Current State of the Art").
  nucleon     N_g(x) = eps_abc (u_a^T C gamma_5 d_b) u_{c,g},  C = gamma_2 gamma_4,
              source N-bar with the same diquark matrix, positive-parity projector
              (1 + gamma_4)/2.  Both Wick terms of the two u lines are kept.

Propagator layout: S[t, z, y, x, sink_spin, sink_colour, src_spin, src_colour].
"""
import numpy as np

from .gamma import GAMMA, GAMMA5, P_MINUS, P_PLUS, CHARGE_C, ID4
from . import dirac

GAMMA_FH = GAMMA[2] @ GAMMA5          # gamma_3 gamma_5
CG5 = CHARGE_C @ GAMMA5               # diquark matrix C gamma_5
PROJ_POS = 0.5 * (ID4 + GAMMA[3])     # (1 + gamma_4)/2

_EPS = np.zeros((3, 3, 3))
for (a, b, c), sgn in {(0, 1, 2): 1, (1, 2, 0): 1, (2, 0, 1): 1,
                       (0, 2, 1): -1, (2, 1, 0): -1, (1, 0, 2): -1}.items():
    _EPS[a, b, c] = sgn


def embed_wall(b4, Ls):
    """P (b at s=0): slice 0 gets P_- b, slice Ls-1 gets P_+ b."""
    out = np.zeros((Ls,) + b4.shape, dtype=np.complex128)
    out[0] = P_MINUS @ b4
    out[Ls - 1] = P_PLUS @ b4
    return out


def inject_source(Ub, b4, p):
    """eta = D(m_f=1) P (b at s=0)."""
    return dirac.mobius(Ub, embed_wall(b4, p.Ls), p, mf=1.0)


def project_4d(y):
    """q = P_- y_0 + P_+ y_{Ls-1}."""
    return P_MINUS @ y[0] + P_PLUS @ y[-1]


def fh_source(S4):
    """Gamma S(z) on every site (Gamma = gamma_3 gamma_5 on the sink spin index).
    S4 is one 4D propagator column [t,z,y,x,spin,colour] or a full propagator
    [t,z,y,x,spin,colour,spin',colour']."""
    if S4.ndim == 6:
        return GAMMA_FH @ S4
    return np.einsum("ij,...jakb->...iakb", GAMMA_FH, S4)


def nucleon_2pt(U1, D, U2):
    """C(t) = sum_x Tr[P+ G(x)] with the two u lines U1, U2 and the d line D:

      G_{g g'} = eps_abc eps_a'b'c' (CG5)_{al be} (CG5b)_{be' al'} *
                 [ U1^{aa'}_{al al'} D^{bb'}_{be be'} U2^{cc'}_{g g'}
                 - U1^{ac'}_{al g'}  D^{bb'}_{be be'} U2^{ca'}_{g al'} ]

    with CG5b = gamma_4 (C gamma_5)^+ gamma_4 the source diquark matrix.  Propagators
    are [t,z,y,x,spin,colour,spin',colour'].  Returns complex C[t]."""
    cg5b = GAMMA[3] @ np.conj(CG5.T) @ GAMMA[3]
    # rearrange to [V, colour, colour', spin, spin']
    def cs(S):
        T = S.shape[0]
        return np.transpose(S, (0, 1, 2, 3, 5, 7, 4, 6)).reshape(T, -1, 3, 3, 4, 4)
    u1, d, u2 = cs(U1), cs(D), cs(U2)
    # diquark-sandwiched d line: Dt^{bb'}_{al, al'} = CG5_{al be} D^{bb'}_{be be'} CG5b_{be' al'}
    dt = np.einsum("ij,tvbcjk,kl->tvbcil", CG5, d, cg5b)
    # direct term: Tr_spin-free pieces
    #   term1_{g g'} = eps eps [sum_{al al'} U1^{aa'}_{al al'} Dt^{bb'}_{al al'}] U2^{cc'}_{g g'}
    #   term2_{g g'} = eps eps sum_{al al'} U1^{ac'}_{al g'} Dt^{bb'}_{al al'} U2^{ca'}_{g al'}
    ee = np.einsum("abc,def->abcdef", _EPS, _EPS)
    t1 = np.einsum("abcdef,tvadij,tvbeij,tvcfgh->tvgh", ee, u1, dt, u2, optimize=True)
    t2 = np.einsum("abcdef,tvafih,tvbeij,tvcdgj->tvgh", ee, u1, dt, u2, optimize=True)
    G = t1 - t2
    return np.einsum("hg,tvgh->t", PROJ_POS, G)


def fh_effective_coupling(c2, c3):
    """Effective coupling from the Feynman-Hellmann correlator (Sec. "Current State of the
    Art": the FH propagator carries the current at every time, so one extra solve gives
    all source-sink separations).  With R(t) = Re[C_FH(t) / C(t)], the derivative of
    log C(t) in the current's coupling, the matrix element is the slope of R at large t:
        g_eff(t) = R(t+1) - R(t),   t = 0 .. T-2.
    c2 = C(t), c3 = C_FH(t) (complex, length T)."""
    r = (np.asarray(c3, dtype=np.complex128) / np.asarray(c2, dtype=np.complex128)).real
    return r[1:] - r[:-1]
