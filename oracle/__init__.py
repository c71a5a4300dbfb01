"""FP64 CPU oracle for resolvent sampling + Rayleigh-Ritz (test infrastructure).

Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline / reference legs
of `bench.py` may import this package.  The product (the CUDA library and its
Python binding) never imports it and shares no code with it.
"""
from .rsrr import (sample_points, quad_weights, inside, eval_fn, assemble,
                   coeff_matrix, resolvent_samples, backward_error_inf,
                   sample_matrix, normalize_columns, truncated_basis, project,
                   ss_full, residual, plain_residual, rsrr, negative_inertia,
                   negative_inertia_band, bisect_real_eigenvalues,
                   argument_principle_count, companion_eigvals,
                   distances, assemble_dense, resolvent_samples_dense, taylor_terms,
                   taylor_coefficients, residual_dense, backward_error_inf_dense, rsrr_dense,
                   argument_principle_count_dense, ShiftPow, assemble_terms,
                   resolvent_samples_terms, backward_error_inf_terms, residual_terms, rsrr_terms,
                   interpolation_weights, moment_matrix, ss_ri, ssrr_m, gauss_legendre,
                   rect_sides, rect_counts, rect_rule, contour_quadrature, contour_path,
                   phase_det_band, RECT_PANEL)
