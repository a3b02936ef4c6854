"""FP64 CPU oracle for the multi-distance holography functional F2 and its gradients.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or link this
package: only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` use it.  It shares no code with the CUDA
path (``paper_2407_20304_gb300``), and it imports nothing from it.

What it computes (Nikitin et al., "X-ray nano-holotomography reconstruction with
simultaneous probe retrieval"):

* ``holo``  - geometry of Sec. 2 (m~_j, omega_j, zeta_j), the Fresnel operator D_z of
  Appendix A (Eq. defPz/defGz), the magnify+shift resample M_{1/m~} S_t of Eq. min1,
  the forward model of Eq. fwd_model_cone3, the amplitude functional F2 (Eq. min1)
  and its gradients (Eq. gradpsi and the probe gradient that follows it).
* ``cg``    - the nonlinear conjugate-gradient iteration of Sec. 2 with the Dai-Yuan
  direction (Eq. DaiYuan2) and a backtracking line search that never increases F.

Every floating-point quantity is float64 / complex128.  All functions are plain
full-grid definitions (no blocking, no fusion, no reordering beyond the formulas).
"""

from . import holo, cg  # noqa: F401
