"""Solver settings of the named workloads (shared by bench.py and the tests; no arithmetic)."""

# Batched uneven workload: 4096 random LTV instances (see workloads.batched_uneven), FP32
# iterations with the FP64 factorisation, accelerated iteration with restart, one launch.
BATCHED_UNEVEN = dict(
    name="batched_uneven_ltv_4096",
    seed=3,
    batch=4096,
    rho=1.0,
    # Stop test c <= eps (Algorithm 1, step 5). c <= 1e-8 leaves about a quarter of the batch
    # (mostly nu/nx >= 0.6) further than 1e-4 from the optimum, in FP64 as in FP32 (the FP64
    # oracle misses on 10 of 48 sampled instances); c <= 1e-12 reaches 1e-4 on all of them in
    # FP64. FP32 iterations level off near c ~ 1e-11..1e-10, where their iterates are already
    # within about 1e-5, so they stop on the stall test (pimpc_set_stall) there.
    eps=1e-12,
    stall_window=100,  # stop when c has not halved for max(window, rel x i0) iterations, i0 the
    stall_rel=0.3,     # first iteration with c <= stall_below (FP32 floor)
    stall_factor=0.5,
    stall_below=1e-9,  # ... counted only once c <= 1e-9 (early plateaus of the accelerated
                       # iteration, far above the floor, do not count)
    max_iters=5000,
    accel=1,
    eta=0.999,
    accuracy=1e-4,     # a solve counts when max|w - w*| / max(1, max|w*|) <= accuracy
    ref_eps=1e-20,     # FP64 reference solve (same GPU) used to score accuracy
    ref_max_iters=20000,
    oracle_score_sample=64,  # instances also scored against the converged FP64 oracle
    polish_iters=2000,  # FP64 polish variant: FP64 iterations after the FP32 ones ...
    polish_eps=1e-13,   # ... until c <= polish_eps
)

# Plain single-instance linear MPC (nx=4, nu=2, N=20), 200 iterations.
PLAIN_LTI = dict(seed=1, nx=4, nu=2, N=20, iters=200)
