"""CPU oracle of the X-SLAM complex-step (CSFD) X-KinectFusion step.

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import, call or execute this package:
only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` use it.

What it is: a plain, slow, obviously correct restatement of X-SLAM (Peng et al., ACM TOG 43(4) 2024)
Sec. 3 (CSFD) and Sec. 4.1 (X-KinectFusion), in numpy with full ``complex128`` arithmetic, h = 1e-20,
one complex run per perturbed parameter ("perturbing variables one by one", Sec. 6). The same code
run on ``float64`` arrays is the uncomplexified pipeline. It shares no code with the CUDA path; the
only common module is the seeded input generator, which holds none of the method's arithmetic.

Modules, in the order of the paper's pipeline:
  csfd      Eq. csfd (Im f(x+hi)/h) and the Sec. 3 worked example f(x) = (e^x + x^3 + x)/(x + 1)
  se3       Eq. lie, rotvector, rotation_jacobi: complex SE(3) exponential; pose read-out
  measure   Sec. 4.1 surface measurement: depth pyramid, Eq. vertex, Eq. normal
  icp       Sec. 4.1 differentiable ICP: Eq. icp, Eq. "icp approx" -> A x = b, pose update
  fusion    Sec. 4.1 surface update: running TSDF average, Eq. bi_interpolate, Psi
  raycast   Sec. 4.1 ray casting: fixed-step march, zero crossing, normal = grad F / |grad F|
  pipeline  the per-frame step and whole-sequence runs with K seeds

Parity status: every function is pinned by tests in tests/test_oracle_*.py against closed forms,
library routines (scipy.linalg.expm), invariants or central finite differences, except the
noisy-trajectory results of the large workloads, which have no closed form ("parity unpinned" for
those end results beyond the oracle itself).
"""
