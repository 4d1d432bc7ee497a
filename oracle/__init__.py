"""Plain, slow CPU oracle for the embedded Sierpinski gasket (test infrastructure).

This package is test infrastructure, not part of the product.  Only the test
suite, ``__graft_entry__.smoke()`` and the CPU-baseline / reference legs of
``bench.py`` may import it.  It shares no code with the CUDA library and never
imports it; inputs come from the separate ``synth`` module.

Everything here follows "Efficient GPU Thread Mapping on Embedded 2D Fractals"
(Navarro, Quezada, Hitschfeld, Vega, Bustos): section numbers, equations and
lemmas are cited in each function.  Floating point is FP64.
"""
from .gasket import (  # noqa: F401
    Domain,
    beta,
    block_table,
    ca_step,
    ca_run,
    diffusion_loss_gradients,
    diffusion_matrix,
    diffusion_run,
    diffusion_step,
    embed,
    grid_dims,
    hash_arith,
    hash_table,
    is_member,
    lambda_canonical,
    lambda_paper,
    member_mask,
    n_members,
    reduce_sum,
    sw_write,
)
from . import nbb  # noqa: F401,E402  (other fractals of the NBB family)
