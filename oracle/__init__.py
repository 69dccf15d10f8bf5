"""FP64 CPU oracle for TV-regularised frequency-domain FWI.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this
package: only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline``
/ ``--impl reference`` legs of ``bench.py`` use it.  It shares no code with
the CUDA library (no kernels, tables, constants or helpers) and is a plain,
slow, obviously correct restatement of the paper (Guo, Auerbach, Eldar,
"TV-Regularized Frequency-Domain Full-Waveform Inversion for Single-Sided
Linear Ultrasound Array Data"):

* ``model``    -- geometry, contrast (Eq. 1-3), wavenumber, SoS inverse map
* ``green``    -- point and cell-integrated Green's functions, offset lattice
* ``operator`` -- Lippmann-Schwinger operator (Eq. 5, Sec. IV-A), incident
                  fields, dense-LU and BiCGSTAB solves
* ``inverse``  -- data (Eq. 4), misfit, adjoint sources / solves, gradient,
                  Jacobian products (Eq. 15-17)
* ``admm``     -- discrete gradient and adjoint, Gauss-Newton m-step
                  (Eq. 9-12), isotropic shrink (Eq. 13-14), dual update,
                  one iteration of Algorithm 1

Every floating-point computation is complex128 / float64.  Where the paper
is silent the reading taken is stated at the function that applies it.
"""
from . import model, green, operator, inverse, admm  # noqa: F401
from .model import Problem  # noqa: F401
