"""Spin-polarised (collinear) exact exchange.

Eq. HF of arXiv 1712.07973 sums over spin channels sigma with per-spin
occupations f_{i,sigma} (Sec. 2, Eq. 1): the channels do not couple, so
E_x = E_x[psi_up, f_up] + E_x[psi_down, f_down] and the action of each
channel's Fock operator uses that channel's orbitals only.  A spin plan is one
plan per channel on the same grid (they share nothing but the kernel choice).
"""

from .exx import ExxPlan

__all__ = ["ExxSpinPlan"]


class ExxSpinPlan:
    """Two-channel plan; occupations per channel (typically f <= 1)."""

    def __init__(self, n, h, alpha, occ_up, occ_down, **kw):
        self.up = ExxPlan(n, h, alpha, occ_up, **kw)
        self.down = ExxPlan(n, h, alpha, occ_down, **kw)

    def energy(self, psi_up, psi_down):
        return self.up.energy(psi_up) + self.down.energy(psi_down)

    def apply(self, psi_up, psi_down):
        """(E_x, Vx psi_up, Vx psi_down)."""
        Eu, vu = self.up.apply(psi_up)
        Ed, vd = self.down.apply(psi_down)
        return Eu + Ed, vu, vd

    def close(self):
        self.up.close()
        self.down.close()
