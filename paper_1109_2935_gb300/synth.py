"""Seeded synthetic inputs: gauge fields, fat/long links and sources.

These stand in for the production gauge configurations of the paper's solver runs
(Sec. 9: a 32^3x256 Wilson-clover ensemble and a 64^3x192 asqtad ensemble), which
are not available. Both the CUDA path and the oracle receive the arrays produced
here; this module holds none of the Dirac-operator, preconditioner or solver
arithmetic. All arrays are natural layout, complex128:
  gauge / fat / long links  [t, z, y, x, mu, 3, 3]
  Wilson spinor             [t, z, y, x, 4, 3]
  staggered spinor          [t, z, y, x, 3]

Random numbers come from a ``torch.Generator`` seeded per field on the requested
device, so a (seed, device) pair always gives the same field.
"""
import torch

_GELL_MANN = None


def _gell_mann(device):
    global _GELL_MANN
    if _GELL_MANN is None or _GELL_MANN.device != torch.device(device):
        l = torch.zeros(8, 3, 3, dtype=torch.complex128)
        l[0, 0, 1] = l[0, 1, 0] = 1
        l[1, 0, 1], l[1, 1, 0] = -1j, 1j
        l[2, 0, 0], l[2, 1, 1] = 1, -1
        l[3, 0, 2] = l[3, 2, 0] = 1
        l[4, 0, 2], l[4, 2, 0] = -1j, 1j
        l[5, 1, 2] = l[5, 2, 1] = 1
        l[6, 1, 2], l[6, 2, 1] = -1j, 1j
        l[7, 0, 0] = l[7, 1, 1] = 1 / 3 ** 0.5
        l[7, 2, 2] = -2 / 3 ** 0.5
        _GELL_MANN = l.to(device)
    return _GELL_MANN


def _gen(seed, device):
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def _cgauss(shape, g, device, scale=1.0):
    re = torch.randn(shape, generator=g, device=device, dtype=torch.float64)
    im = torch.randn(shape, generator=g, device=device, dtype=torch.float64)
    return torch.complex(re, im) * scale


def reunitarize(U):
    """Gram-Schmidt on rows 1-2, row 3 = conj(row1 x row2): the nearest-by-construction
    SU(3) matrix."""
    a = U[..., 0, :]
    a = a / torch.linalg.vector_norm(a, dim=-1, keepdim=True)
    b = U[..., 1, :]
    b = b - (a.conj() * b).sum(-1, keepdim=True) * a
    b = b / torch.linalg.vector_norm(b, dim=-1, keepdim=True)
    c = torch.linalg.cross(a, b).conj()
    return torch.stack([a, b, c], dim=-2)


def su3_exp_gaussian(shape, sigma, g, device):
    """exp(i H) with H = sum_a w_a lambda_a / 2, w_a ~ N(0, sigma^2), re-unitarised."""
    w = torch.randn(tuple(shape) + (8,), generator=g, device=device, dtype=torch.float64) * sigma
    H = torch.einsum("...a,aij->...ij", w.to(torch.complex128), _gell_mann(device)) * 0.5
    flat = H.reshape(-1, 3, 3)
    out = torch.empty_like(flat)
    step = 1 << 20
    for i in range(0, flat.shape[0], step):
        out[i:i + step] = torch.linalg.matrix_exp(1j * flat[i:i + step])
    return reunitarize(out.reshape(H.shape))


def haar_su3(shape, g, device):
    """Haar-distributed SU(3): Gram-Schmidt of two complex-Gaussian rows, row 3 from
    their cross product."""
    z = _cgauss(tuple(shape) + (3, 3), g, device)
    return reunitarize(z)


def _roll(U, mu, n):
    """Field at x + n*mu for natural [t, z, y, x, ...] arrays (periodic)."""
    return torch.roll(U, shifts=-n, dims=3 - mu)


def smooth(U, alpha=0.5, steps=3):
    """APE-like smoothing, all four directions updated simultaneously:
    U' = reunit[(1 - alpha) U_mu(x) + alpha/6 sum_{nu != mu} (upper + lower staple)]."""
    for _ in range(steps):
        new = torch.empty_like(U)
        for mu in range(4):
            Umu = U[..., mu, :, :]
            st = torch.zeros_like(Umu)
            for nu in range(4):
                if nu == mu:
                    continue
                Unu = U[..., nu, :, :]
                Unu_xpmu = _roll(Unu, mu, 1)
                Umu_xpnu = _roll(Umu, nu, 1)
                st = st + Unu @ Umu_xpnu @ Unu_xpmu.conj().transpose(-1, -2)
                Unu_xmnu = _roll(Unu, nu, -1)
                Umu_xmnu = _roll(Umu, nu, -1)
                Unu_xmnu_pmu = _roll(Unu_xmnu, mu, 1)
                st = st + Unu_xmnu.conj().transpose(-1, -2) @ Umu_xmnu @ Unu_xmnu_pmu
            new[..., mu, :, :] = reunitarize((1 - alpha) * Umu + (alpha / 6.0) * st)
        U = new
    return U


def wilson_gauge(dims, sigma, smear_steps, seed, device="cpu"):
    """Random SU(3) links exp(i sigma-Gaussian) followed by ``smear_steps`` smoothing
    steps. ``dims = (LX, LY, LZ, LT)``."""
    LX, LY, LZ, LT = dims
    g = _gen(seed, device)
    U = su3_exp_gaussian((LT, LZ, LY, LX, 4), sigma, g, device)
    if smear_steps:
        U = smooth(U, 0.5, smear_steps)
    return U.contiguous()


def asqtad_links(dims, seed_fat, seed_long, device="cpu"):
    """Fat links: complex Gaussian entries scaled by 1/8 (not unitary). Long links:
    Haar SU(3)."""
    LX, LY, LZ, LT = dims
    fat = _cgauss((LT, LZ, LY, LX, 4, 3, 3), _gen(seed_fat, device), device, 1.0 / 8.0)
    long = haar_su3((LT, LZ, LY, LX, 4), _gen(seed_long, device), device)
    return fat.contiguous(), long.contiguous()


def wilson_spinor(dims, seed, device="cpu"):
    LX, LY, LZ, LT = dims
    return _cgauss((LT, LZ, LY, LX, 4, 3), _gen(seed, device), device).contiguous()


def staggered_spinor(dims, seed, device="cpu", parity=None):
    """Gaussian 3-complex source; with ``parity`` set, zero on the other parity."""
    LX, LY, LZ, LT = dims
    s = _cgauss((LT, LZ, LY, LX, 3), _gen(seed, device), device)
    if parity is not None:
        t = torch.arange(LT, device=device).view(LT, 1, 1, 1)
        z = torch.arange(LZ, device=device).view(1, LZ, 1, 1)
        y = torch.arange(LY, device=device).view(1, 1, LY, 1)
        x = torch.arange(LX, device=device).view(1, 1, 1, LX)
        mask = ((t + z + y + x) % 2 == parity)
        s = s * mask[..., None]
    return s.contiguous()


def unit_gauge(dims, device="cpu"):
    LX, LY, LZ, LT = dims
    U = torch.zeros((LT, LZ, LY, LX, 4, 3, 3), dtype=torch.complex128, device=device)
    U[..., 0, 0] = U[..., 1, 1] = U[..., 2, 2] = 1
    return U


def gauge_transform(U, G, hop=1):
    """U'_mu(x) = G(x) U_mu(x) G(x + hop*mu)^dagger for G of shape [t, z, y, x, 3, 3]
    (hop = 3 for the long links, which join x to x + 3 mu)."""
    out = torch.empty_like(U)
    for mu in range(4):
        out[..., mu, :, :] = G @ U[..., mu, :, :] @ _roll(G, mu, hop).conj().transpose(-1, -2)
    return out


def ptc_weights(channels, seed, noise=0.05):
    """Initial weights of a parallel-transport convolution network with the given
    channel list: each layer passes channel 0 through on the local path (identity spin
    matrix) plus complex Gaussian entries of standard deviation `noise` everywhere, so no
    hidden channel starts dead. Complex128 tensors shaped (9, c_out, c_in, 4, 4)."""
    g = _gen(seed, "cpu")
    out = []
    for l in range(len(channels) - 1):
        shape = (9, channels[l + 1], channels[l], 4, 4)
        W = _cgauss(shape, g, "cpu", noise)
        W[0, 0, 0] += torch.eye(4, dtype=W.dtype)
        out.append(W)
    return out
