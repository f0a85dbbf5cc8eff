"""torch.autograd access to the band-energy adjoint of the C ABI.

``band_energy(system, S_vals, H_vals, z, w)`` returns the band energy E as a
0-d tensor; ``backward`` gives dE/dS_vals and dE/dH_vals (the stored entries
of the block layout, taken as independent entries) from the gradients that
``tb_band_energy`` computes in the same solve.  The arithmetic runs in the
library; this module only moves arguments and scales the saved gradients by
the incoming gradient.
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
