"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

This module holds none of the compression method's arithmetic: it only draws random numbers
and builds the matrices that the compression is applied to. Both the oracle and the CUDA path
consume its outputs; neither side imports the other.

Workloads (the paper's own test operators need codes and data that are not available, so these
stand in for them):

* ``log_kernel``: the 2D logarithmic kernel A_ij = log|x_i - x_j| (A_ii = 0) on N points evenly
  spaced in angle on the closed curve r(theta) = 1 + 0.3 cos(5 theta), ordered along the curve.
  A smooth-curve kernel of the boundary-integral type used in Section 5.1; it is only
  approximately HBS.
* ``exact_hbs``: an HBS matrix of exact block rank k (Section 3.2) in classical form: random
  orthonormal leaf bases (m x k) and parent bases (2k x k), Gaussian sibling couplings B (k x k)
  and Gaussian leaf diagonal blocks. Its telescoping factors (Section 3.3) are returned too, with
  parent blocks D_tau = [[0, B_ab], [B_ba, 0]]; the dense matrix is assembled block by block from
  expanded bases, not through the apply algorithm.
* ``double_layer``: the Nystrom (trapezoid) matrix of the boundary integral equation of Section
  5.1, (1/2) I + K with the double-layer kernel on the same curve (a second operator of the kind
  the paper compresses; the paper's own contour is only in a figure).
* ``gaussian``: i.i.d. N(0, 1) arrays from numpy's PCG64 (used where test matrices are passed
  in as inputs rather than drawn by the method's own counter-based generator).

The tree used by ``exact_hbs`` is the one of Section 3.1 (ceil split, split while a node is
larger than the leaf threshold); it is rebuilt here from that description.
"""

from .generators import (CurvePoints, ExactHBS, curve_points, double_layer, double_layer_rows,
                         double_layer_torch, exact_hbs, exact_hbs_packed_torch,
                         gaussian, log_kernel, log_kernel_rows, log_kernel_torch, pack_telescoping,
                         packed_layout, seed_for)

__all__ = ["CurvePoints", "ExactHBS", "curve_points", "double_layer", "double_layer_rows",
           "double_layer_torch", "exact_hbs", "exact_hbs_packed_torch",
           "gaussian", "log_kernel", "log_kernel_rows", "log_kernel_torch", "pack_telescoping",
           "packed_layout", "seed_for"]
