"""CPU oracle for robust proton planning by ADMM-BB (Fu, Taasti, Zarepisheh).

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
CPU-baseline leg may import this package.  The product path (the CUDA library
and its Python binding) never imports, links or calls it, and this package
never imports the product: the two share no code.  Inputs come from the
separate `synthetic` generator.

Everything is plain float64 NumPy/SciPy, slow and written to be checked
against the paper by eye:

  problem.py    scenario objective and its gradient (Sec. 2.1, Eqs. 1-2, 4),
                weighted matrices of App. A, default parameters
  admm_bb.py    ADMM with Barzilai-Borwein dual step (Sec. 2.2, Eqs. 5-8),
                subproblem by cached Cholesky (App. A) or by CG
  pgd.py        projected gradient descent with Armijo search (Sec. 2.1, Eq. 3)
  exact.py      the exact box-constrained optimum: brute-force KKT enumeration
                and a library bounded least-squares solve, plus certificates
  boyd.py       textbook scaled-form consensus ADMM, written separately, which
                ADMM-BB must reproduce when the BB step is switched off
  quantize.py   the reduced-precision storage form (per-column FP32 scale,
                bfloat16 or FP8-e4m3 codes) as a plain definition
  mlp.py        the learned warm start's network: forward pass, MSE loss and
                its gradient by the chain rule (float64)
  dose_constraints.py
                linear dose limits (maximum, minimum, mean) as extra ADMM
                blocks (Sec. 4 names them; the splitting is a reading) and the
                exact constrained optimum by active-set enumeration

Readings where the paper is silent or garbled (each one is a parameter):
  * z-update: z = P(mean_s(x_s + y_s/rho)) by default ("std"); the paper's
    printed form P(mean_s x_s) is zmode="lit".
  * the Armijo test is sufficient decrease, f(x+) <= f(x) + b g'(x+ - x);
    the printed inequality has the wrong direction.
  * the fixed rho is used in the x-subproblem, the z-update and the dual
    residual; the BB step replaces rho only in the dual update.
"""
from .problem import Weighted, default_rho, lipschitz  # noqa: F401
from .admm_bb import admm_bb  # noqa: F401
from .pgd import pgd  # noqa: F401
from .exact import kkt_bruteforce, lsq_box, box_qp_newton, normal_equations, certificates  # noqa: F401
from .boyd import consensus_admm_scaled  # noqa: F401
from .quantize import quantised_problem, quantise_values, bf16_round, e4m3_round  # noqa: F401
from .dose_constraints import DoseConstraint, constraint_rows, admm_bb_constrained, kkt_bruteforce_lin  # noqa: F401
