"""FP64 CPU oracle for the moment-encoded (HOME-LBM) multi-level lattice.

TEST INFRASTRUCTURE ONLY.  This package is the slow, plain reference that the
CUDA path is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.
The product package ``paper_2603_14982_gb300`` never imports it, and this
package never imports the product package: the two share no code.

Modules (each function cites the passage of the paper it follows):

* ``lattice``      D3Q27 velocity set, weights, Hermite basis, the third-order
                   reconstruction f_i(M) (Eq. three_order_f) and the moment
                   projection (Eq. rho_u_stress).
* ``single_level`` one pull-stream + moment-space collision step on a dense grid
                   (Sec. 3.1 "Collision and Streaming", Sec. 4 mixture tau).
* ``hierarchy``    the declarative block hierarchy (Sec. 5.1, Sec. 6.1, Sec. 6.3,
                   Eq. level-selection Phi).
* ``multilevel``   Algorithm 1 with downward/upward transfers and the S^neq
                   rescaling (Sec. 5.2, Eq. upload_S, Eq. downward_rescale).
* ``coupling``     the coupled finest-level step of Fig. 4 (streaming only,
                   drag exchange, collision; Sec. 5.4).
* ``deposit``      solid fraction, fluid fraction and drag force per finest
                   node from particle counts (Sec. 4, Sec. 5.4).
* ``adjoint``      reverse-mode gradients of the single-level step and of the
                   multi-level advance (no counterpart in the paper).

Arithmetic is float64 (complex128 for complex-step derivative checks).  Arrays
are indexed [z, y, x]; a moment field is a tensor of shape (10, nz, ny, nx) with
rows (rho, u_x, u_y, u_z, S_xx, S_yy, S_zz, S_xy, S_xz, S_yz).
"""
