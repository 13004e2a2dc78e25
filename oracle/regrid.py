"""Restart with a change of resolution (oracle).

Test infrastructure only (see the package docstring).

Sec. 2.1 states that the spatial resolution can be changed at every restart
by interpolation and mode padding.  The paper gives no formulas; the reading
taken here:
* radial: the unique polynomial of degree <= Nr_src - 1 through the source's
  nodal values (Chebyshev-Gauss-Lobatto nodes of the same gap), evaluated at
  the target's nodes -- written in the Lagrange product form, one basis
  polynomial per source node.  The wall nodes of both grids coincide, so wall
  values are copied exactly;
* Fourier: coefficients of modes present in both runs are copied, modes only
  the target has are zero (padding), modes only the source has are dropped
  (truncation).  The same gap (eta) and axial period (Lz) are required;
* temperature: a source without T given to a target with T gets the target's
  discrete conductive profile in the (0,0) mode; a target without T drops it.
The divergence of the interpolated field is that of an interpolant, not zero
on the target's discrete operators; the first stage of the next step projects
it.
"""
from __future__ import annotations

import numpy as np

from .grid import cgl_radii


def lagrange_matrix(x_src: np.ndarray, x_dst: np.ndarray) -> np.ndarray:
    """P[i, s] = l_s(x_dst[i]), l_s the Lagrange basis polynomial of node s."""
    n = len(x_src)
    P = np.empty((len(x_dst), n))
    for i, x in enumerate(x_dst):
        for s in range(n):
            v = 1.0
            for t in range(n):
                if t != s:
                    v *= (x - x_src[t]) / (x_src[s] - x_src[t])
            P[i, s] = v
    return P


def regrid(X_src: np.ndarray, eta: float, mdl) -> np.ndarray:
    """State of another resolution -> state on ``mdl``'s grid.

    X_src: complex (nf_src, Nr_src, M_src+1, 2 K_src+1), axial index in FFT
    order (0..K, -K..-1).  Returns complex (mdl.nf, Nr, M+1, 2K+1).
    """
    nf_src, Nr_src, M1, NK_src = X_src.shape
    K_src = (NK_src - 1) // 2
    P = lagrange_matrix(cgl_radii(Nr_src, eta), mdl.g.r)
    Nr, M, K = mdl.g.Nr, mdl.M, mdl.K
    out = np.zeros((mdl.nf, Nr, M + 1, 2 * K + 1), dtype=complex)
    mk = min(M, M1 - 1)
    kc = min(K, K_src)
    for f in range(min(nf_src, mdl.nf)):
        for m in range(mk + 1):
            for k in range(-kc, kc + 1):
                col = X_src[f, :, m, k % NK_src]          # FFT-order index of k
                out[f, :, m, k % (2 * K + 1)] = P @ col
    if mdl.nf == 4 and nf_src == 3:
        out[3, :, 0, 0] = mdl.base[3, :, 0, 0]
    return out
