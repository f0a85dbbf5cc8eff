"""torch.autograd access to the adjoints of the C ABI.

``band_energy(system, S_vals, H_vals, z, w)`` returns the band energy E as a
0-d tensor; ``backward`` gives dE/dS_vals and dE/dH_vals (the stored entries
of the block layout, taken as independent entries) from the gradients that
``tb_band_energy`` computes in the same solve.

``mulliken_charges(system, S_vals, H_vals, z, w)`` returns the gross Mulliken
populations (per atom, or per orbital with ``per_orbital=True``); its
``backward`` turns the incoming gradient into orbital weights v (an atom's
weight on each of its orbitals) and asks ``tb_mulliken_vjp`` for
dL/dH_vals and dL/dS_vals of L = sum_a v_a q_a, the vector-Jacobian product
of the populations.  Only orbitals with a nonzero weight are solved, so the
gradient of a few atoms' charges is cheap on any system size.

The arithmetic runs in the library; this module only moves arguments and
scales the gradients by the incoming gradient.
"""
from __future__ import annotations

import numpy as np

from . import tb


class BandEnergy:
    """Namespace for the autograd.Function (built lazily so that importing
    the package does not import torch)."""
    _fn = None

    @classmethod
    def function(cls):
        if cls._fn is None:
            import torch

            class _BandEnergy(torch.autograd.Function):
                @staticmethod
                def forward(ctx, S_vals, H_vals, structure, z, w, g_s, opts):
                    orb, brow, bcol = structure
                    h = tb.tb_create(orb, brow, bcol, S_vals.detach().cpu().numpy(),
                                     H_vals.detach().cpu().numpy(), None, 0.0)
                    E, gH, gS, _ = tb.tb_band_energy(h, z, w, g_s, opts=opts, n_values=S_vals.numel())
                    h.close()
                    ctx.save_for_backward(torch.as_tensor(gS, dtype=S_vals.dtype, device=S_vals.device),
                                          torch.as_tensor(gH, dtype=H_vals.dtype, device=H_vals.device))
                    return torch.tensor(E, dtype=S_vals.dtype, device=S_vals.device)

                @staticmethod
                def backward(ctx, grad_E):
                    gS, gH = ctx.saved_tensors
                    return grad_E * gS, grad_E * gH, None, None, None, None, None

            cls._fn = _BandEnergy
        return cls._fn


def band_energy(structure, S_vals, H_vals, z, w, g_s=2.0, opts=None):
    """E(S_vals, H_vals) with autograd.  ``structure`` = (orb_per_atom,
    brow_ptr, bcol) of the block layout; S_vals and H_vals are float64
    tensors of the stored entries (both triangles, as tb_create takes them)."""
    return BandEnergy.function().apply(S_vals, H_vals, tuple(np.asarray(a) for a in structure), z, w, g_s,
                                       opts)


class MullikenCharges:
    """Namespace for the autograd.Function of the Mulliken populations."""
    _fn = None

    @classmethod
    def function(cls):
        if cls._fn is None:
            import torch

            class _Mulliken(torch.autograd.Function):
                @staticmethod
                def forward(ctx, S_vals, H_vals, structure, z, w, g_s, opts, per_orbital):
                    orb, brow, bcol = structure
                    h = tb.tb_create(orb, brow, bcol, S_vals.detach().cpu().numpy(),
                                     H_vals.detach().cpu().numpy(), None, 0.0)
                    if per_orbital:
                        q, _ = tb.tb_mulliken_orbital(h, z, w, np.arange(h.n_orb, dtype=np.int32), g_s, opts=opts)
                    else:
                        q, _ = tb.tb_mulliken_charges(h, z, w, g_s, opts=opts)
                    # the handle stays for the backward solves (closed there,
                    # or by its finaliser if no gradient is asked for)
                    ctx.h, ctx.orb, ctx.z, ctx.w, ctx.g_s, ctx.opts = h, np.asarray(orb), z, w, g_s, opts
                    ctx.per_orbital, ctx.n_values = per_orbital, S_vals.numel()
                    ctx.dev, ctx.dtype = S_vals.device, S_vals.dtype
                    return q.to(device=S_vals.device, dtype=S_vals.dtype)

                @staticmethod
                @torch.autograd.function.once_differentiable
                def backward(ctx, grad_q):
                    g = grad_q.detach().to(dtype=torch.float64).cpu().numpy()
                    v = g if ctx.per_orbital else np.repeat(g, ctx.orb)
                    gH, gS, _ = tb.tb_mulliken_vjp(ctx.h, ctx.z, ctx.w, np.ascontiguousarray(v), ctx.n_values,
                                                   ctx.g_s, opts=ctx.opts)
                    ctx.h.close()
                    return (torch.as_tensor(gS, dtype=ctx.dtype, device=ctx.dev),
                            torch.as_tensor(gH, dtype=ctx.dtype, device=ctx.dev), None, None, None, None, None, None)

            cls._fn = _Mulliken
        return cls._fn


def mulliken_charges(structure, S_vals, H_vals, z, w, g_s=2.0, opts=None, per_orbital=False):
    """Gross Mulliken populations q(S_vals, H_vals) with autograd: per atom
    (default) or per orbital.  ``structure`` = (orb_per_atom, brow_ptr, bcol)
    of the block layout; S_vals and H_vals are float64 tensors of the stored
    entries (both triangles, as tb_create takes them)."""
    return MullikenCharges.function().apply(S_vals, H_vals, tuple(np.asarray(a) for a in structure), z, w, g_s,
                                            opts, per_orbital)
