// hydro_device.cuh -- per-cell and per-face device arithmetic of the update.
//
// Pieces of one unsplit finite-volume step of the compressible Euler
// equations (gamma-law gas, constant gravity): boundary index mapping, the
// MC-limited PLM slope, the MUSCL-Hancock half step in primitive variables,
// the HLLC face flux, and the CTA-level max reduction.  T is double or float.
//
// Hydrostatic-background mode (HSE): the stored state is U' = U - U0(z).
// Primitives hold (rho', u, p'); totals are rho = rho0 + rho', p = p0 + p'.
// Face fluxes carry p' in the normal momentum; the background's discrete
// imbalance B_k enters the momentum update as a source.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#include "hydro_internal.h"
#include "pieces.h"

namespace hydro {

// Interior source index of coordinate g along an axis of n cells (n >= 2),
// for g in [-2, n+1]; flip is set for a mirror image (reflecting boundary).
// On a halo side (slab decomposition, z only) g in [-2, -1] or [n, n+1] is
// returned as is: those planes are stored in the buffer.
// Coordinates further out (cells of a ragged tile beyond the domain, whose
// results are never stored) are clamped into range.
template <bool HALO = false>
__device__ __forceinline__ int map_index(int g, int n, int bclo, int bchi, bool &flip)
{
    flip = false;
    // a halo side (z only): the two planes beyond the slab are stored next to it
    if constexpr (HALO)
        if ((g < 0 && bclo == BC_HALO) || (g >= n && bchi == BC_HALO)) return g;
    if (g < 0) {
        if (bclo == BC_PERIODIC) g += n;
        else if (bclo == BC_REFLECT) { g = -1 - g; flip = true; }
        else g = 0;
    } else if (g >= n) {
        if (bchi == BC_PERIODIC) g -= n;
        else if (bchi == BC_REFLECT) { g = 2 * n - 1 - g; flip = true; }
        else g = n - 1;
    }
    return min(max(g, 0), n - 1);
}

// ---- Row vectors for the staging loads.  A haloed tile row whose x range
// lies inside the grid is fetched as aligned vectors of W cells (16 bytes:
// float4 / double2; or 8 bytes: float2) instead of one 4- or 8-byte load per
// cell: vector k of the row covers the cells x0 - W + W k .. x0 - 1 + W k,
// TX / W + 2 vectors in all, so the row's halo of depth 2 is covered (with
// W = 4 also the two cells beyond it on each side, which lie in the same
// 32-byte sectors as the halo cells).  Two adjacent cells -- a pair -- are
// then written to shared memory as one 8- or 16-byte store.
template <typename T, int W> struct RowVec;
template <> struct RowVec<float, 4> { using V = float4; };
template <> struct RowVec<float, 2> { using V = float2; };
template <> struct RowVec<double, 2> { using V = double2; };

template <typename T, int W>
__device__ __forceinline__ T vec_lane(const typename RowVec<T, W>::V &v, int e)
{
    return reinterpret_cast<const T *>(&v)[e];   // e a compile-time constant: a register
}

template <typename T, int W>
__device__ __forceinline__ typename RowVec<T, W>::V ld_vec(const T *p)
{
    return __ldg(reinterpret_cast<const typename RowVec<T, W>::V *>(p));
}

// Whether the rows of a tile starting at x0, TX cells wide, can be fetched
// as vectors of W cells: the state's base and variable planes aligned to a
// vector (nx a multiple of W, so every row is), and the vectors' x range
// [x0 - W, x0 + TX + W) inside [0, nx) -- no x boundary mapping in the halo.
template <typename T, int TX, int W>
__device__ __forceinline__ bool rows_vectorisable(const void *U, int nx, long long vs, int x0)
{
    static_assert(TX % W == 0, "tile width a multiple of the vector width");
    constexpr unsigned long long align = W * sizeof(T);
    return (reinterpret_cast<unsigned long long>(U) & (align - 1)) == 0 && nx % W == 0 && vs % W == 0 &&
           x0 >= W && x0 + TX + W <= nx;
}

// Reciprocal square root, quotient and reciprocal in the working precision.
// FP64 uses CUDA's IEEE-accurate double routines; FP32 uses the SFU
// approximations (rsqrtf, __fdividef: at most 2 ulp), well inside the FP32
// path's error budget.
__device__ __forceinline__ double rsqrt_t(double x) { return rsqrt(x); }
__device__ __forceinline__ float rsqrt_t(float x) { return rsqrtf(x); }

// FP64 reciprocal by Newton-Raphson iteration on f(y) = 1/y - b, which
// doubles the number of correct bits per step: y <- y + y (1 - b y).  The
// start value is the hardware approximation rcp.approx.ftz.f64 (about 20
// correct bits), so two steps reach the FP64 rounding level; the result is
// within a couple of ulp of 1/b for normal b (not always correctly rounded),
// far inside the 1e-10 parity budget.  Costs one SFU operation and four
// FMAs on the FP64 pipe.
__device__ __forceinline__ double rcp_t(double b)
{
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(b));
    double e = fma(-b, y, 1.0);
    y = fma(y, e, y);
    e = fma(-b, y, 1.0);
    return fma(y, e, y);
}
__device__ __forceinline__ float rcp_t(float b) { return __fdividef(1.0f, b); }
__device__ __forceinline__ double div_t(double a, double b) { return a * rcp_t(b); }
__device__ __forceinline__ float div_t(float a, float b) { return __fdividef(a, b); }

// Conserved -> primitive pieces of the staging conversion with every
// rounding spelled out (explicit multiplies and fused multiply-adds): the
// compiler then has no contraction choices, so each staging path (row
// vectors or mapped cells, in whichever kernel) gives the same bits.
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }

// p = (gamma - 1)(E - |m|^2 / (2 rho)) from the momentum components m, the
// velocities u = m / rho, the total energy e and gm1 = gamma - 1: |m|^2 / rho
// as u . m summed in axis order, then (gamma - 1) fma(-1/2, u . m, E).
template <typename T, int ND>
__device__ __forceinline__ T pressure_of(const T (&m)[ND], const T (&u)[ND], T e, T gm1)
{
    T k = mul_rn(u[0], m[0]);
#pragma unroll
    for (int d = 1; d < ND; ++d) k = fma_rn(u[d], m[d], k);
    return mul_rn(gm1, fma_rn(T(-0.5), k, e));
}

// A step constant in the kernel's precision: the FP64 value, or its FP32
// copy rounded on the host (the same value as a device-side conversion).
template <typename T>
__device__ __forceinline__ T arg_t(double d, float f)
{
    if constexpr (sizeof(T) == 4) return f;
    else return d;
}

// First item of a CTA-strided loop (i = start, start + NT, ...) whose items
// past the first NT -- a second pass for a few threads -- should land on
// warps 2, 3, ... instead of 0, 1, ...: each SM sub-partition (warp mod 4)
// has its own FP64 unit and issue slot, and when two loops of a phase both
// leave their second pass on warp 0, that sub-partition is the critical
// path.  Covers the same items as start = tid.
template <int NT>
__device__ __forceinline__ int rotated_start(int tid)
{
    return NT >= 128 ? (tid + NT - 64) % NT : tid;
}

// x > 0 (false for +-0 and for negative values).  For doubles the test is
// an integer test of the bit pattern, which keeps it off the FP64 pipe.
__device__ __forceinline__ bool positive(double x) { return __double_as_longlong(x) > 0; }
__device__ __forceinline__ bool positive(float x) { return x > 0.0f; }
// x / 2 of a non-negative x.  For doubles an exact halving on the integer
// pipe (one off the exponent field; the same bits as 0.5 * x for normal
// results) rather than on the FP64 pipe: 0 for x below 2^-1021, where the
// half would not be normal; infinities and NaNs are passed through.
__device__ __forceinline__ double half_nonneg(double x)
{
    const long long b = __double_as_longlong(x);
    const long long h = b >= (2ll << 52) ? b - (1ll << 52) : 0ll;
    return __longlong_as_double(b >= (0x7ffll << 52) ? b : h);
}
__device__ __forceinline__ float half_nonneg(float x) { return 0.5f * x; }
// Sign tests for the HLLC fan branches: x >= 0 and x <= 0 as numeric
// comparisons (both zeros satisfy both), done on the bit pattern for doubles:
// x >= 0 holds for a clear sign bit and for -0 (whose pattern is the most
// negative 64-bit integer); x <= 0 holds for a set sign bit and for +0.
// A wave speed S* of -0 (reached at reflecting walls, where the two states
// are mirror images) therefore takes the left branch, as S* = +0 does.
__device__ __forceinline__ bool nonnegative(double x)
{
    const long long b = __double_as_longlong(x);
    return b >= 0 || b == (long long)0x8000000000000000ull;
}
__device__ __forceinline__ bool nonnegative(float x) { return x >= 0.0f; }
__device__ __forceinline__ bool nonpositive(double x) { return __double_as_longlong(x) <= 0; }
__device__ __forceinline__ bool nonpositive(float x) { return x <= 0.0f; }

// Minimum and maximum.  FP64: by the order of integer keys of the bit
// patterns (a sign-magnitude to two's-complement map that orders all
// non-NaN doubles, -0 below +0), on the integer pipe rather than the FP64
// pipe that bounds the FP64 step; FP32: the hardware min/max.
__device__ __forceinline__ long long order_key(double x)
{
    const long long b = __double_as_longlong(x);
    return b ^ ((b >> 63) & 0x7fffffffffffffffll);
}
__device__ __forceinline__ double min_t(double a, double b) { return order_key(a) <= order_key(b) ? a : b; }
__device__ __forceinline__ double max_t(double a, double b) { return order_key(a) >= order_key(b) ? a : b; }
__device__ __forceinline__ float min_t(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ float max_t(float a, float b) { return fmaxf(a, b); }

// MC limiter (van Leer 1977): full-cell slope sign(dr) min(2|dl|, 2|dr|,
// |dl+dr|/2) when dl and dr have the same sign, else 0.
__device__ __forceinline__ float mc_slope(float dl, float dr)
{
    const float a = fminf(2.0f * fminf(fabsf(dl), fabsf(dr)), 0.5f * fabsf(dl + dr));
    return (dl * dr > 0.0f) ? copysignf(a, dr) : 0.0f;
}

// FP64 form: the sign test, both minima, the doubling and the halving act
// on the IEEE bit patterns (integer pipe; for non-negative doubles integer
// order is numeric order, and adding or removing 1 in the exponent field
// multiplies a normal number by 2 or 1/2 exactly), leaving the differences
// and dl + dr on the FP64 pipe.  When dl and dr share a sign both are
// nonzero and their sum is nonzero; a |dl + dr| below 2^-1021 (no normal
// halving) gives a zero slope.
__device__ __forceinline__ double mc_slope(double dl, double dr)
{
    constexpr long long ABS = 0x7fffffffffffffffll, ONE_EXP = 1ll << 52;
    const long long bl = __double_as_longlong(dl), br = __double_as_longlong(dr);
    const long long al = bl & ABS, ar = br & ABS;
    const bool same = ((bl ^ br) >= 0) && al != 0 && ar != 0;
    const long long m = min(al, ar);
    const long long twice = m < (0x7fell << 52) ? m + ONE_EXP : m;       // 2 min(|dl|, |dr|)
    const long long as = __double_as_longlong(dl + dr) & ABS;
    const long long half = as >= (2ll << 52) ? as - ONE_EXP : 0ll;        // |dl + dr| / 2
    const double a = __longlong_as_double(min(twice, half));
    return same ? copysign(a, dr) : 0.0;
}

// CFL signal speed of a cell, sum_d (|u_d| + c) / dx_d, from its momenta m
// (ND components), rinv = 1/rho and sound speed c, arranged as
// (sum_d |m_d| / dx_d) / rho + c sum_d 1/dx_d (the sum of the 1/dx_d is
// loop-invariant in the callers).
template <typename T, int ND>
__device__ __forceinline__ T signal_speed(const T *m, T rinv, T c, const T (&inv_dx)[3])
{
    T a = fabs(m[0]) * inv_dx[0];
    T sidx = inv_dx[0];
#pragma unroll
    for (int d = 1; d < ND; ++d) {
        a = fma(fabs(m[d]), inv_dx[d], a);
        sidx += inv_dx[d];
    }
    return fma(rinv, a, c * sidx);
}

// Background seen by one cell in HSE mode (all zero in plain mode).
template <typename T>
struct CellBG {
    T rho, p;            // centre
    T drho, dp, B;       // z differences across the cell and imbalance
    T rho_lo, p_lo;      // low z face
    T rho_hi, p_hi;      // high z face
};

template <typename T, bool HSE>
__device__ __forceinline__ CellBG<T> cell_bg(const PlaneBGT<T> *bg, int k)
{
    CellBG<T> b;
    if constexpr (HSE) {
        const PlaneBGT<T> &c = bg[k + 2];
        const PlaneBGT<T> &u = bg[k + 3];
        b.rho = c.rho_c; b.p = c.p_c;
        b.drho = c.drho; b.dp = c.dp; b.B = c.B;
        b.rho_lo = c.rho_f; b.p_lo = c.p_f;
        b.rho_hi = u.rho_f; b.p_hi = u.p_f;
    } else {
        b.rho = b.p = b.drho = b.dp = b.B = T(0);
        b.rho_lo = b.p_lo = b.rho_hi = b.p_hi = T(0);
    }
    return b;
}

// The face densities and pressures c -/+ dw_d / 2 of a cell (c: the cell's
// half-step or centre state) into rp[d] = {rho_lo, rho_hi, p_lo, p_hi}, and
// whether all of them are positive once the background is added back (HSE:
// the face tables along z).  In plain mode the FP64 path skips the addition
// of the zero background (0 + x is not folded for doubles); the FP32 path
// keeps it (its measured instruction schedule).
template <typename T, int ND, bool HSE>
__device__ __forceinline__ bool face_rho_p_positive(const T (&c)[ND + 2], const T (&dw)[ND][ND + 2],
                                                    const CellBG<T> &bg, T (&rp)[ND][4])
{
    constexpr int NV = ND + 2;
    constexpr bool BGADD = HSE || sizeof(T) == 4;
    bool ok = true;
#pragma unroll
    for (int d = 0; d < ND; ++d) {
        T rb_lo = bg.rho, rb_hi = bg.rho, pb_lo = bg.p, pb_hi = bg.p;
        if (HSE && d == 2) { rb_lo = bg.rho_lo; rb_hi = bg.rho_hi; pb_lo = bg.p_lo; pb_hi = bg.p_hi; }
        rp[d][0] = c[0] - T(0.5) * dw[d][0];
        rp[d][1] = c[0] + T(0.5) * dw[d][0];
        rp[d][2] = c[NV - 1] - T(0.5) * dw[d][NV - 1];
        rp[d][3] = c[NV - 1] + T(0.5) * dw[d][NV - 1];
        const T r_lo = BGADD ? rb_lo + rp[d][0] : rp[d][0];
        const T r_hi = BGADD ? rb_hi + rp[d][1] : rp[d][1];
        const T p_lo = BGADD ? pb_lo + rp[d][2] : rp[d][2];
        const T p_hi = BGADD ? pb_hi + rp[d][3] : rp[d][3];
        ok = ok && positive(r_lo) && positive(r_hi) && positive(p_lo) && positive(p_hi);
    }
    return ok;
}

// MUSCL-Hancock half step (Toro, 3rd ed., sec. 14.4) in primitive variables
// for one cell: wh = w - (dt/2) sum_d A_d(w) dw_d / dx_d + (dt/2) S(w), where
// S(w) is gravity on the velocities.  On return dw holds the slopes used
// (all zero after the positivity fallback) and the face states are
// wh -/+ dw_d / 2; their densities and pressures, formed for the positivity
// test, are returned in rp[d] = {rho_lo, rho_hi, p_lo, p_hi} (the same
// values: the caller takes them instead of forming them again).  Returns
// true when the fallback was taken.
template <typename T, int ND, bool HSE, bool GZ = false, bool RINV = false>
__device__ __forceinline__ bool hancock(const T (&w)[ND + 2], T (&dw)[ND][ND + 2],
                                        T (&wh)[ND + 2], T (&rp)[ND][4], T hdt, const T (&inv_dx)[3],
                                        T gam, const T (&grav)[3], const CellBG<T> &bg,
                                        T rinv_given = T(0))
{
    constexpr int NV = ND + 2;
    const T rho = HSE ? bg.rho + w[0] : w[0];
    const T pr = HSE ? bg.p + w[NV - 1] : w[NV - 1];
    // RINV: 1/rho as computed when the cell was staged (the same value)
    const T rinv = RINV ? rinv_given : rcp_t(rho);
    const T gp = gam * pr;
    // A_d(w) dw_d / dx_d summed over d: rho: u_d drho_d + rho du_{d,d};
    // u_e: u_d du_{e,d} (+ dp_d / rho for e = d); p: u_d dp_d + gamma p du_{d,d}.
    // The rho and p rows take their normal-velocity terms through one
    // divergence, div u = sum_d du_{d,d} / dx_d; 1/dx_d is folded into the
    // other coefficients.
    T divu = dw[0][1] * inv_dx[0];
#pragma unroll
    for (int d = 1; d < ND; ++d) divu = fma(dw[d][1 + d], inv_dx[d], divu);
    T rate[NV];
    rate[0] = -rho * divu;
#pragma unroll
    for (int e = 0; e < ND; ++e) rate[1 + e] = T(0);
    rate[NV - 1] = -gp * divu;
#pragma unroll
    for (int d = 0; d < ND; ++d) {
        const T un_dx = w[1 + d] * inv_dx[d];
        const T rinv_dx = rinv * inv_dx[d];
        rate[0] = fma(-un_dx, dw[d][0], rate[0]);
#pragma unroll
        for (int e = 0; e < ND; ++e) rate[1 + e] = fma(-un_dx, dw[d][1 + e], rate[1 + e]);
        rate[1 + d] = fma(-rinv_dx, dw[d][NV - 1], rate[1 + d]);
        rate[NV - 1] = fma(-un_dx, dw[d][NV - 1], rate[NV - 1]);
    }
    // gravity on the velocities: g rho'/rho - B/rho in HSE mode, g otherwise
    T gsrc[ND];
#pragma unroll
    for (int d = 0; d < ND; ++d) gsrc[d] = HSE ? grav[d] * (w[0] * rinv) : grav[d];
    if constexpr (HSE) {
        const T wz = w[3];
        rate[0] -= wz * bg.drho * inv_dx[2];
        rate[4] -= wz * bg.dp * inv_dx[2];
        gsrc[2] -= bg.B * rinv;
    }
    // (GZ: gravity along the last axis only -- the other axes' zero terms
    // are not added)
#pragma unroll
    for (int d = 0; d < ND; ++d)
        if (!GZ || d == ND - 1) rate[1 + d] += gsrc[d];
#pragma unroll
    for (int q = 0; q < NV; ++q) wh[q] = w[q] + hdt * rate[q];

    // positivity of every predicted face density and pressure
    const bool ok = face_rho_p_positive<T, ND, HSE>(wh, dw, bg, rp);
    if (!ok) {
#pragma unroll
        for (int d = 0; d < ND; ++d)
#pragma unroll
            for (int q = 0; q < NV; ++q) dw[d][q] = T(0);
#pragma unroll
        for (int q = 0; q < NV; ++q) wh[q] = w[q];
#pragma unroll
        for (int d = 0; d < ND; ++d)
            if (!GZ || d == ND - 1) wh[1 + d] += hdt * gsrc[d];
#pragma unroll
        for (int d = 0; d < ND; ++d) {
            rp[d][0] = rp[d][1] = w[0];
            rp[d][2] = rp[d][3] = w[NV - 1];
        }
    }
    return !ok;
}

// Face state q of axis d (hi: the high face) of a cell after hancock or
// mol_faces (there with wh = w): the density and pressure as returned in rp,
// the velocities wh -/+ dw_d / 2.
template <typename T, int ND>
__device__ __forceinline__ T face_value(int q, int d, bool hi, const T (&wh)[ND + 2], const T (&dw)[ND][ND + 2],
                                        const T (&rp)[ND][4])
{
    if (q == 0) return rp[d][hi ? 1 : 0];
    if (q == ND + 1) return rp[d][hi ? 3 : 2];
    return hi ? wh[q] + T(0.5) * dw[d][q] : wh[q] - T(0.5) * dw[d][q];
}

// Face states of the method of lines (no predictor): w -/+ dw_d / 2, with
// the same positivity fallback as the half step (every slope of the cell
// zeroed when a face density or pressure would not be positive); rp as in
// hancock.
template <typename T, int ND, bool HSE>
__device__ __forceinline__ void mol_faces(const T (&w)[ND + 2], T (&dw)[ND][ND + 2], const CellBG<T> &bg,
                                          T (&rp)[ND][4])
{
    constexpr int NV = ND + 2;
    if (!face_rho_p_positive<T, ND, HSE>(w, dw, bg, rp)) {
#pragma unroll
        for (int d = 0; d < ND; ++d) {
#pragma unroll
            for (int q = 0; q < NV; ++q) dw[d][q] = T(0);
            rp[d][0] = rp[d][1] = w[0];
            rp[d][2] = rp[d][3] = w[NV - 1];
        }
    }
}

// Piecewise parabolic face values (Colella and Woodward 1984, uniform grid)
// of the cell with value a, face neighbours am and ap and MC-limited slopes
// sm, s, sp (cells i-1, i, i+1): interface values (a + a')/2 - (s' - s)/6,
// then the parabola limited to be monotone: flat at a local extremum, else
// a face value moved so that the parabola has no interior extremum.
template <typename T>
__device__ __forceinline__ void ppm_faces(T am, T a, T ap, T sm, T s, T sp, T &lo, T &hi)
{
    const T sixth = T(1.0 / 6.0);
    T aL = T(0.5) * (am + a) - (s - sm) * sixth;
    T aR = T(0.5) * (a + ap) - (sp - s) * sixth;
    const bool flat = (aR - a) * (a - aL) <= T(0);
    const T da = aR - aL;
    const T a6 = T(6) * (a - T(0.5) * (aL + aR));
    const T dd = da * da, d6 = da * a6;
    const bool fix_l = !flat && d6 > dd;
    const bool fix_r = !flat && !fix_l && -dd > d6;
    lo = flat ? a : (fix_l ? T(3) * a - T(2) * aR : aL);
    hi = flat ? a : (fix_r ? T(3) * a - T(2) * aL : aR);
}

// HLLC flux along axis D (Toro, 3rd ed., sec. 10.4-10.6) with Davis wave
// speeds S_L = min(u_L - c_L, u_R - c_R), S_R = max(u_L + c_L, u_R + c_R).
// wl, wr hold (rho', u, p') and (rb, pb) the background at the face; in plain
// mode rb = pb = 0.  The normal momentum flux carries p' (= p in plain mode).
// Branches: 0 <= S_L -> F_L; S_L < 0 <= S* -> F*_L; S* < 0 < S_R -> F*_R;
// S_R <= 0 -> F_R.  igm1 = 1/(gamma - 1).
//
// Arithmetic is arranged to need two square-root reciprocals and two
// divisions per face: c = g rsqrt(g rho) with g = gamma p.  The star state of
// Toro eq. (10.39), rho*_K = rho_K (S_K - u_K) / (S_K - S*) with velocity
// (S*, v_t) and E*_K = rho*_K [E_K / rho_K + (S* - u_K)(S* + p_K / (rho_K (S_K - u_K)))],
// enters only through F*_K = F_K + S_K (U*_K - U_K), whose components reduce
// to multiples of one factor h = S_K (S* - u_K) / (S_K - S*):
//   S_K (rho*_K - rho_K)             = rho_K h                      (= c0)
//   S_K (rho*_K v_t - rho_K v_t)     = c0 v_t
//   S_K (rho*_K S* - rho_K u_K)      = S_K c0
//   S_K (E*_K - E_K)                 = h (E_K + p_K + m_K S*),  m_K = rho_K (S_K - u_K)
// (rho*_K - rho_K = rho_K (S* - u_K) / (S_K - S*); the energy line follows
// from E*_K - E_K written over the common denominator S_K - S*).
template <typename T, int ND, int D, bool HSE>
__device__ __forceinline__ void hllc(const T (&wl)[ND + 2], const T (&wr)[ND + 2], T rb, T pb,
                                     T gam, T igm1, T (&f)[ND + 2])
{
    constexpr int NV = ND + 2;
    const T rl = HSE ? rb + wl[0] : wl[0];
    const T rr = HSE ? rb + wr[0] : wr[0];
    const T pl = HSE ? pb + wl[NV - 1] : wl[NV - 1];
    const T pr = HSE ? pb + wr[NV - 1] : wr[NV - 1];
    const T ul = wl[1 + D], ur = wr[1 + D];
    const T gpl = gam * pl, gpr = gam * pr;
    const T cl = gpl * rsqrt_t(gpl * rl);
    const T cr = gpr * rsqrt_t(gpr * rr);
    // S_L - u_L = min(-c_L, (u_R - u_L) - c_R) and S_R - u_R = max(c_L - (u_R - u_L), c_R):
    // the offsets the star factors m_K = rho_K (S_K - u_K) need, and S_L, S_R from them
    const T du = ur - ul;
    const T al = min_t(-cl, du - cr);
    const T ar = max_t(cl - du, cr);
    const T sl = ul + al, sr = ur + ar;

    // Branch-free: every face computes S* and the star correction and the
    // branch of the HLLC fan is applied by selects.  The chosen branch's
    // values are the same as with branches, and the straight-line code lets
    // a thread's independent faces interleave.  S* and 1/(S_K - S*) are
    // finite for positive densities and pressures (S_L < u_L, S_R > u_R).
    const T dpp = wr[NV - 1] - wl[NV - 1];   // background cancels in the difference
    const T ml = rl * al, mr = rr * ar;
    const T sstar = div_t(dpp + ml * ul - mr * ur, ml - mr);
    const bool sup_l = nonnegative(sl);     // whole fan moves right: F_L
    const bool sup_r = nonpositive(sr);     // whole fan moves left: F_R
    const bool left = sup_l || (!sup_r && nonnegative(sstar));
    const bool star = !sup_l && !sup_r;
    const T rk = left ? rl : rr;
    const T pk = left ? pl : pr;
    const T ppk = left ? wl[NV - 1] : wr[NV - 1];
    const T sk = left ? sl : sr;
    const T mk = left ? ml : mr;
    T vk[ND];
#pragma unroll
    for (int e = 0; e < ND; ++e) vk[e] = left ? wl[1 + e] : wr[1 + e];
    const T uk = vk[D];
    T ke = T(0);
#pragma unroll
    for (int e = 0; e < ND; ++e) ke += vk[e] * vk[e];
    // E_K + p_K = p_K gamma / (gamma - 1) + rho_K |v_K|^2 / 2
    const T hk = fma(pk, igm1 + T(1), rk * half_nonneg(ke));

    // Euler flux of the chosen side
    const T mflux = rk * uk;
    f[0] = mflux;
#pragma unroll
    for (int e = 0; e < ND; ++e) f[1 + e] = mflux * vk[e];
    f[1 + D] += ppk;
    f[NV - 1] = uk * hk;

    // F*_K = F_K + S_K (U*_K - U_K), applied only inside the fan
    const T h = (sk * rcp_t(sk - sstar)) * (sstar - uk);
    const T c0 = rk * h;                    // S_K (rho*_K - rho_K)
    const T fE = fma(h, fma(mk, sstar, hk), f[NV - 1]);
    if constexpr (sizeof(T) == 8) {
        // FP64 (bound by its FP64 pipe): each star component formed by one
        // fused multiply-add onto F_K (or one addition) and selected
        f[0] = star ? f[0] + c0 : f[0];
#pragma unroll
        for (int e = 0; e < ND; ++e) {
            const T fs = (e == D) ? fma(sk, c0, f[1 + e]) : fma(c0, vk[e], f[1 + e]);
            f[1 + e] = star ? fs : f[1 + e];
        }
        f[NV - 1] = star ? fE : f[NV - 1];
    } else {
        const T cs = star ? c0 : T(0);
        f[0] += cs;
#pragma unroll
        for (int e = 0; e < ND; ++e) f[1 + e] = fma(cs, (e == D) ? sk : vk[e], f[1 + e]);
        f[NV - 1] = star ? fE : f[NV - 1];
    }
}

// Mirror image of a face state across a wall normal to axis D.
template <typename T, int NV, int D>
__device__ __forceinline__ void mirror_state(const T (&src)[NV], T (&dst)[NV])
{
#pragma unroll
    for (int q = 0; q < NV; ++q) dst[q] = src[q];
    dst[1 + D] = -src[1 + D];
}

// Max over the CTA of a double (every thread passes its value; the result is
// valid in thread 0).  red must hold 32 doubles.
template <int NT>
__device__ __forceinline__ double block_max(double v, double *red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (warp == 0) {
        v = lane < NT / 32 ? red[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    }
    return v;
}

// The same max taken in the working precision (max is exact in any
// precision), widened to FP64 once: an FP32 step keeps the reduction off the
// FP64 pipe.  red must hold 32 doubles.
template <int NT, typename T>
__device__ __forceinline__ double block_max_t(T v, double *red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    T *r = reinterpret_cast<T *>(red);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) r[warp] = v;
    __syncthreads();
    if (warp == 0) {
        v = lane < NT / 32 ? r[lane] : T(0);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    }
    return double(v);
}

// Last-CTA finalisation of a step's time control.  Each of the nblocks
// contributions (CTAs, or work items of one instance) calls it once with its
// max signal speed (valid in thread 0), whether any of its cells failed the
// admissibility check, and its slot `part` in a.partial, after storing its
// part of the new state.
// The CTA that arrives last takes the grid maximum (max is exact, so arrival
// order does not matter), commits the error bits, sets the next dt in FP64
// and advances time.  advance = false only recomputes dt (initialisation).
// Only this CTA writes the fields that every CTA reads at kernel start, and
// it does so after all CTAs have read them.
template <int NT>
__device__ __forceinline__ void finish_step(double smax_cta, bool bad_cta, const StepArgs &a,
                                            int nblocks, int part, double dt_used, bool advance,
                                            int *s_last)
{
    if (threadIdx.x == 0) {
        if (bad_cta) atomicOr(&a.ctrl->err_new, 1);
        a.partial[part] = smax_cta;
        __threadfence();
        const unsigned prev = atomicAdd(&a.ctrl->counter, 1u);
        *s_last = (prev == (unsigned)(nblocks - 1));
    }
    __syncthreads();
    if (!*s_last) return;
    __threadfence();
    double m = 0.0;
    for (int i = threadIdx.x; i < nblocks; i += NT) m = fmax(m, __ldcg(a.partial + i));
    __shared__ double red2[32];
    m = block_max<NT>(m, red2);
    if (threadIdx.x == 0) {
        Ctrl *C = a.ctrl;
        if (advance) {
            const double t = C->t;
            C->t = (dt_used >= a.t_end - t) ? a.t_end : t + dt_used;
            C->dt_last = dt_used;
            C->step = C->step + 1;
        }
        int e = atomicExch(&C->err_new, 0);
        if (!(m > 0.0) || !isfinite(m)) e |= 1;
        C->err |= e;
        C->max_speed = m;
        C->dt_next = m > 0.0 ? a.cfl / m : 0.0;
        C->counter = 0u;
        __threadfence();
    }
}

// Next work item of a persistent batched launch from list L of the queue
// for this launch's parity (valid in every thread), or -1 when the list is
// exhausted.  The CTA that is last to find the list exhausted resets the
// counters (every other CTA has stopped claiming by then), so the next
// launch of this parity starts from item 0.  Every thread must call it.
__device__ __forceinline__ int claim_item(BatchQueue *q, int L, int parity, int *s_it)
{
    if (threadIdx.x == 0) {
        const int n = q->nitems[L];
        int it = (int)atomicAdd(&q->next[L][parity], 1u);
        if (it >= n) {
            it = -1;
            if (atomicAdd(&q->exited[L][parity], 1u) == gridDim.x - 1) {
                q->next[L][parity] = 0u;
                q->exited[L][parity] = 0u;
                __threadfence();
            }
        }
        *s_it = it;
    }
    __syncthreads();
    return *s_it;
}

}  // namespace hydro
