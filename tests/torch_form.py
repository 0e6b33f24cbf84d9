"""FP64 torch-ops formulation of the PW source terms (test helper).

Whole-array PyTorch CPU operations: periodic x/y neighbours by ``torch.roll``,
vertical neighbours by shifting with zero fill, the per-level coefficients
broadcast along z, and the levels the method does not compute multiplied by
zero.  Listing 1 (Sec. 2.1) for su, the same pattern on the staggered grid for
sv and sw.  Written independently of the oracle (no shared code); its use is
the cross-check the oracle gets from a second formulation, and -- through
torch autograd -- an adjoint that owes nothing to the hand-derived gather.
Fields are [nx, ny, nz] float64 tensors; coefficient tables are 0-based per
level.
"""
import torch


def _at(a, di=0, dj=0, dk=0):
    """a at (i+di, j+dj, k+dk): periodic in i and j, zero beyond the column."""
    if di or dj:
        a = torch.roll(a, shifts=(-di, -dj), dims=(0, 1))
    if dk == 1:
        a = torch.cat([a[..., 1:], torch.zeros_like(a[..., :1])], dim=-1)
    elif dk == -1:
        a = torch.cat([torch.zeros_like(a[..., :1]), a[..., :-1]], dim=-1)
    return a


def source_terms(u, v, w, tcx, tcy, tzc1, tzc2, tzd1, tzd2):
    nz = u.shape[-1]
    c1, c2 = torch.as_tensor(tzc1, dtype=u.dtype), torch.as_tensor(tzc2, dtype=u.dtype)
    d1, d2 = torch.as_tensor(tzd1, dtype=u.dtype), torch.as_tensor(tzd2, dtype=u.dtype)
    # su: x, y and vertical terms (the top level has no upper flux: u(k+1) is zero there)
    su = tcx * (_at(u, -1) * (u + _at(u, -1)) - _at(u, 1) * (u + _at(u, 1))) \
        + tcy * (_at(u, 0, -1) * (_at(v, 0, -1) + _at(v, 1, -1)) - _at(u, 0, 1) * (v + _at(v, 1))) \
        + c1 * _at(u, 0, 0, -1) * (_at(w, 0, 0, -1) + _at(w, 1, 0, -1)) \
        - c2 * _at(u, 0, 0, 1) * (w + _at(w, 1))
    sv = tcx * (_at(v, -1) * (_at(u, -1) + _at(u, -1, 1)) - _at(v, 1) * (u + _at(u, 0, 1))) \
        + tcy * (_at(v, 0, -1) * (v + _at(v, 0, -1)) - _at(v, 0, 1) * (v + _at(v, 0, 1))) \
        + c1 * _at(v, 0, 0, -1) * (_at(w, 0, 0, -1) + _at(w, 0, 1, -1)) \
        - c2 * _at(v, 0, 0, 1) * (w + _at(w, 0, 1))
    sw = tcx * (_at(w, -1) * (_at(u, -1) + _at(u, -1, 0, 1)) - _at(w, 1) * (u + _at(u, 0, 0, 1))) \
        + tcy * (_at(w, 0, -1) * (_at(v, 0, -1) + _at(v, 0, -1, 1)) - _at(w, 0, 1) * (v + _at(v, 0, 0, 1))) \
        + d1 * _at(w, 0, 0, -1) * (w + _at(w, 0, 0, -1)) \
        - d2 * _at(w, 0, 0, 1) * (w + _at(w, 0, 0, 1))
    m_uv = torch.ones(nz, dtype=u.dtype)
    m_uv[0] = 0.0
    m_w = m_uv.clone()
    m_w[-1] = 0.0
    return su * m_uv, sv * m_uv, sw * m_w


def adjoint_by_autograd(u, v, w, dsu, dsv, dsw, coeffs):
    """J(u,v,w)^T (dsu, dsv, dsw) by reverse-mode autograd of ``source_terms``."""
    x = [torch.as_tensor(a, dtype=torch.float64).clone().requires_grad_(True) for a in (u, v, w)]
    out = source_terms(*x, *coeffs)
    lam = [torch.as_tensor(a, dtype=torch.float64) for a in (dsu, dsv, dsw)]
    torch.autograd.backward(out, lam)
    return tuple(t.grad.numpy() for t in x)
