"""CPU FP64 oracle of the equilibrium projection (test infrastructure, not the product).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU baseline leg may import this
package.  It shares no code with the CUDA path: plain numpy/scipy in float64, each function
citing the passage of the paper (Zhou, Lebensohn, Reischig, Ludwig, Bhattacharya, "Imposing
equilibrium on measured 3-D stress fields using Hodge decomposition and FFT-based optimization")
that it follows.

Conventions (shared with the library boundary, stated here independently):
  * a field is an array ``(6, nz, ny, nx)``, x fastest, Voigt order (xx, yy, zz, yz, xz, xy);
  * tensor index 0/1/2 = x/y/z; array axis -1/-2/-3 = x/y/z;
  * the tensor inner product A:B = sum_ij A_ij B_ij, so off-diagonal Voigt entries weigh 2;
  * forward DFT unnormalised with exp(-2 pi i m.x/N), inverse with exp(+...) and 1/(nx ny nz).

Parity status: every function below is pinned by a ``-m "not gpu"`` test against something other
than itself (brute-force constrained least squares, the paper's printed 25-point stencil,
real-space central differences, closed forms, invariants, an independent library FFT).
"""
from .transforms import dft_axis_direct, dft3_direct, dft3_naive, fft3, ifft3
from .operators import (wavevector, wavevector_grids, biharmonic_symbol_paper,
                        central_diff, stencil25_apply)
from .projection import (project, project_large, project_literal, project_spectrum, divergence,
                         divergence_central_diff, norms, norms_large, inner, frob2)
from .fields import beltrami_field, symgrad_field, smooth_potential, inc_central_diff
from .brute import project_bruteforce
from .hodge import project_compat, hodge_potential
from .grains import grain_means, grain_average
from .padding import project_padded

__all__ = [
    "dft_axis_direct", "dft3_direct", "dft3_naive", "fft3", "ifft3",
    "wavevector", "wavevector_grids", "biharmonic_symbol_paper", "central_diff",
    "stencil25_apply", "project", "project_large", "norms_large", "project_literal",
    "project_spectrum", "divergence",
    "divergence_central_diff", "norms", "inner", "frob2", "beltrami_field", "symgrad_field",
    "smooth_potential", "inc_central_diff", "project_bruteforce", "project_compat",
    "hodge_potential", "grain_means", "grain_average", "project_padded",
]
