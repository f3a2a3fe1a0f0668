"""Seeded synthetic inputs shared by the oracle tests, the CUDA parity tests and bench.py.

This module holds no arithmetic of the solver: it only draws random numbers and
shapes them into the user layouts that both sides accept.

User layouts (all complex128, C order):
  gauge links   U[t, z, y, x, mu, a, b]        U_mu(x) on the link x -> x+mu_hat,
                                               mu = 0,1,2,3 for x,y,z,t
  4D spinor     psi[t, z, y, x, spin, colour]
  5D spinor     psi[s, t, z, y, x, spin, colour]
  batches add a leading right-hand-side axis.

Gauge recipe (synthetic stand-in for the paper's gauge ensembles, Sec. "Performance
Measurement Method"): for every link, a 3x3 complex matrix A with Re, Im ~ N(0,1) is
drawn from numpy Generator(Philox(seed)) in (t, z, y, x, mu, row, col, re/im) order;
H = (A + A^dagger)/2 - tr(.)/3; U = exp(i eps H) by eigendecomposition; U is then
reunitarised (Gram-Schmidt on rows 0 and 1, row 2 = conj(row0 x row1)).
"""
import numpy as np

__all__ = ["gauge_links", "gaussian_spinor5d", "point_source4d", "z2_source4d",
           "random_su3", "lattice_volume"]


def lattice_volume(dims):
    X, Y, Z, T = dims
    return X * Y * Z * T


def _rng(seed):
    return np.random.Generator(np.random.Philox(int(seed)))


def random_su3(n, eps, rng):
    """n SU(3) matrices exp(i eps H), H traceless Hermitian with Gaussian entries."""
    g = rng.standard_normal((n, 3, 3, 2))
    a = g[..., 0] + 1j * g[..., 1]
    h = 0.5 * (a + np.conj(np.swapaxes(a, -1, -2)))
    tr = np.trace(h, axis1=-2, axis2=-1).real / 3.0
    h = h - tr[:, None, None] * np.eye(3)[None]
    w, v = np.linalg.eigh(h)
    u = np.einsum("nij,nj,nkj->nik", v, np.exp(1j * eps * w), np.conj(v))
    # reunitarise
    r0 = u[:, 0, :]
    r0 = r0 / np.linalg.norm(r0, axis=-1, keepdims=True)
    r1 = u[:, 1, :]
    r1 = r1 - np.sum(np.conj(r0) * r1, axis=-1, keepdims=True) * r0
    r1 = r1 / np.linalg.norm(r1, axis=-1, keepdims=True)
    r2 = np.conj(np.cross(r0, r1))
    return np.stack([r0, r1, r2], axis=1)


def gauge_links(dims, eps, seed, chunk=1 << 20):
    """Links U[t,z,y,x,mu,3,3] (complex128) for lattice dims=(X,Y,Z,T)."""
    X, Y, Z, T = dims
    n = X * Y * Z * T * 4
    rng = _rng(seed)
    out = np.empty((n, 3, 3), dtype=np.complex128)
    for i in range(0, n, chunk):
        m = min(chunk, n - i)
        out[i:i + m] = random_su3(m, eps, rng)
    return out.reshape(T, Z, Y, X, 4, 3, 3)


def gaussian_spinor5d(dims, Ls, seed, nrhs=None):
    """Complex Gaussian 5D field [s,t,z,y,x,4,3] (or [nrhs, ...])."""
    X, Y, Z, T = dims
    shape = (Ls, T, Z, Y, X, 4, 3)
    if nrhs is not None:
        shape = (nrhs,) + shape
    g = _rng(seed).standard_normal(shape + (2,))
    return g[..., 0] + 1j * g[..., 1]


def point_source4d(dims, spin, colour, site=(0, 0, 0, 0)):
    """Unit point source at site=(x,y,z,t) in one spin-colour component."""
    X, Y, Z, T = dims
    b = np.zeros((T, Z, Y, X, 4, 3), dtype=np.complex128)
    x, y, z, t = site
    b[t, z, y, x, spin, colour] = 1.0
    return b


def z2_source4d(dims, seed):
    """Real +-1 noise in every (site, spin, colour) component of a 4D source."""
    X, Y, Z, T = dims
    r = _rng(seed).integers(0, 2, size=(T, Z, Y, X, 4, 3))
    return (1.0 - 2.0 * r).astype(np.complex128)


def gaussian_spinor5d_device(dims, Ls, seed, nrhs=1, device="cuda"):
    """Complex Gaussian 5D field [nrhs, s, t, z, y, x, 4, 3] drawn on the GPU with a seeded
    torch Philox generator (for lattices whose complex128 fields do not fit host memory
    comfortably).  Deterministic for a given seed, device type and torch version."""
    import torch
    X, Y, Z, T = dims
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    shape = (nrhs, Ls, T, Z, Y, X, 4, 3, 2)
    r = torch.randn(shape, generator=g, device=device, dtype=torch.float64)
    return torch.view_as_complex(r)


class DeviceSites:
    """Read-only numpy view of selected sites of a device field: field[..., t, z, y, x, :, :]
    with integer index arrays fetches only those sites (what oracle.sample's gather does)."""

    def __init__(self, tensor):
        self.t = tensor

    def __getitem__(self, idx):
        import torch
        if not (isinstance(idx, tuple) and idx[0] is Ellipsis):
            raise IndexError("expected field[..., t, z, y, x, :, :]")
        t, z, y, x = (torch.as_tensor(a, device=self.t.device) for a in idx[1:5])
        return self.t[..., t, z, y, x, :, :].cpu().numpy()


def gauge_links_device(dims, eps, seed, device="cuda", chunk=1 << 16):
    """Links [t,z,y,x,mu,3,3] (complex128, on the GPU) from the recipe of gauge_links, with
    the Gaussian entries drawn by a seeded torch Philox generator on the device instead of
    numpy and exp(i eps H) by the batched matrix exponential (for lattices whose host
    generation would take minutes)."""
    import torch
    X, Y, Z, T = dims
    n = X * Y * Z * T * 4
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    out = torch.empty((n, 3, 3), dtype=torch.complex128, device=device)
    eye = torch.eye(3, dtype=torch.complex128, device=device)
    for i in range(0, n, chunk):
        m = min(chunk, n - i)
        r = torch.randn((m, 3, 3, 2), generator=g, device=device, dtype=torch.float64)
        a = torch.view_as_complex(r)
        h = 0.5 * (a + a.conj().transpose(-1, -2))
        tr = torch.diagonal(h, dim1=-2, dim2=-1).sum(-1).real / 3.0
        h = h - tr[:, None, None] * eye
        u = torch.linalg.matrix_exp(1j * eps * h)   # exp(i eps H), batched on the device
        r0 = u[:, 0, :] / torch.linalg.vector_norm(u[:, 0, :], dim=-1, keepdim=True)
        r1 = u[:, 1, :] - (r0.conj() * u[:, 1, :]).sum(-1, keepdim=True) * r0
        r1 = r1 / torch.linalg.vector_norm(r1, dim=-1, keepdim=True)
        r2 = torch.linalg.cross(r0, r1).conj()
        out[i:i + m] = torch.stack([r0, r1, r2], dim=1)
    return out.reshape(T, Z, Y, X, 4, 3, 3)
