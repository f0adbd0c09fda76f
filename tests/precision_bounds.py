"""Error bounds of the reduced-precision forms, from their storage precision.

Used by the GPU tests that compare FP32 and BF16-deviation runs with the FP64
oracle.  Every bound is a formula of the run (steps N, velocities per cell nv,
velocity-cell volume dv, cells, lid speed U_W) and of the storage format; none
is fitted to a measured error.

FP32.  A step rounds each value at most six times (four operations of the
flux-form streaming, two of the relaxation), each time by 2^-24 of operands
no larger than the local max|f|, and the initial state is rounded once.  With
every rounding of the same sign (no cancellation at all) a moment drifts by at
most eps = (6 N + 1) 2^-24 of its sum of absolute terms: n and the total mass
by eps, U by eps <|c|> (<|c|> = sqrt(pi)/2 for a 2D Maxwellian at theta = 1),
theta = (2/3)(E/n - U^2) by 2 eps.

BF16 deviation.  d = f - M_abs is stored with stochastic rounding: a store
errs by at most one ulp, 2^-7 |d|, with zero mean and standard deviation at
most half an ulp, 2^-8 |d|, independently across velocities.  One step thus
adds to a cell's n an error of standard deviation s_n = sqrt(nv) 2^-8 max|d| dv
and to its n U one of s_u = sqrt(nv) 2^-8 max|c d| dv.  Streaming carries each
step's errors away from the cell at the mean particle speed, hop = <|c|> dt/dx
cells per step, so after k steps they are spread over about pi (hop k)^2
cells; summing the variances, a cell's accumulated error has a standard
deviation at most spread s with spread^2 = sum_{k<=N} 1 / max(1, pi (hop k)^2).
The bounds are six standard deviations.  The total mass, whose errors do not
spread out, gets 6 sqrt(N cells) s_n dx^2.  The deviations of a lid-driven
cavity are bounded by the lid: |M(U) - M(0)| <= 2 |c| U_W M(c) <= 2 U_W
max(|c| e^{-c^2}) / pi = 0.273 U_W and |c (M(U) - M(0))| <= 2 U_W max(c^2
e^{-c^2}) / pi = 0.234 U_W, plus the density and temperature changes of order
Mach^2 (times max M = 1/pi) and the seeded perturbation (amplitude times 1/pi).
"""
import math

U32 = 2.0 ** -24
MEAN_SPEED_2D = math.sqrt(math.pi) / 2


def f32(steps: int) -> dict:
    """Relative bounds (n, theta, total mass) and the bound on |U| error."""
    eps = (6 * steps + 1) * U32
    return {"n": eps, "theta": 2 * eps, "mass": eps, "u": eps * MEAN_SPEED_2D}


def cavity_max_d(uw: float, mach: float, amp: float) -> tuple[float, float]:
    """(max|d|, max|c d|) of a lid-driven cavity with lid speed uw."""
    return 0.273 * uw + (mach ** 2 + amp) / math.pi, 0.234 * uw + 5.0 * (mach ** 2 + amp) / math.pi


def spread(steps: int, hop: float) -> float:
    return math.sqrt(sum(1.0 / max(1.0, math.pi * (hop * k) ** 2) for k in range(1, steps + 1)))


def bf16(steps: int, nv: int, dv: float, cells: int, dx: float, dt: float, uw: float, mach: float,
         amp: float) -> dict:
    """Bounds on n (absolute, n ~ 1), U (absolute), theta (absolute) and the
    total mass (relative to cells dx^2, the mass at n = 1)."""
    md, mcd = cavity_max_d(uw, mach, amp)
    s_n = math.sqrt(nv) * 2.0 ** -8 * md * dv
    s_u = math.sqrt(nv) * 2.0 ** -8 * mcd * dv
    k = 6 * spread(steps, MEAN_SPEED_2D * dt / dx)
    return {"n": k * s_n, "u": k * s_u, "theta": (2 / 3) * 2.5 * k * s_n,
            "mass": 6 * math.sqrt(steps * cells) * s_n / cells}
