"""Solver settings of the named workloads (shared by bench.py and the tests; no arithmetic)."""

# Batched uneven workload: 4096 random LTV instances (see workloads.batched_uneven), FP32
# iterations with the FP64 factorisation, accelerated iteration with restart, one launch.
BATCHED_UNEVEN = dict(
    name="batched_uneven_ltv_4096",
    seed=3,
    batch=4096,
    rho=1.0,
    eps=1e-8,          # stop test c <= eps (Algorithm 1, step 5)
    max_iters=4000,
    accel=1,
    eta=0.999,
    accuracy=1e-4,     # a solve counts when max|w - w*| / max(1, max|w*|) <= accuracy
    ref_eps=1e-15,     # FP64 reference solve (same GPU) used to score accuracy
    ref_max_iters=40000,
    polish_iters=2000,  # FP64 polish variant: FP64 iterations after the FP32 ones ...
    polish_eps=1e-13,   # ... until c <= polish_eps
)

# Plain single-instance linear MPC (nx=4, nu=2, N=20), 200 iterations.
PLAIN_LTI = dict(seed=1, nx=4, nu=2, N=20, iters=200)
