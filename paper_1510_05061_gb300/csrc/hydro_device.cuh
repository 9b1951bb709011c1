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

namespace hydro {

// Interior source index of coordinate g along an axis of n cells (n >= 2),
// for g in [-2, n+1]; flip is set for a mirror image (reflecting boundary).
// Coordinates further out (cells of a ragged tile beyond the domain, whose
// results are never stored) are clamped into range.
__device__ __forceinline__ int map_index(int g, int n, int bclo, int bchi, bool &flip)
{
    flip = false;
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

// MC limiter (van Leer 1977): full-cell slope sign(dr) min(2|dl|, 2|dr|,
// |dl+dr|/2) when dl and dr have the same sign, else 0.
template <typename T>
__device__ __forceinline__ T mc_slope(T dl, T dr)
{
    T a = fmin(fmin(T(2) * fabs(dl), T(2) * fabs(dr)), T(0.5) * fabs(dl + dr));
    return (dl * dr > T(0)) ? copysign(a, dr) : T(0);
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
__device__ __forceinline__ CellBG<T> cell_bg(const PlaneBG *bg, int k)
{
    CellBG<T> b;
    if constexpr (HSE) {
        const PlaneBG &c = bg[k + 2];
        const PlaneBG &u = bg[k + 3];
        b.rho = T(c.rho_c); b.p = T(c.p_c);
        b.drho = T(c.drho); b.dp = T(c.dp); b.B = T(c.B);
        b.rho_lo = T(c.rho_f); b.p_lo = T(c.p_f);
        b.rho_hi = T(u.rho_f); b.p_hi = T(u.p_f);
    } else {
        b.rho = b.p = b.drho = b.dp = b.B = T(0);
        b.rho_lo = b.p_lo = b.rho_hi = b.p_hi = T(0);
    }
    return b;
}

// MUSCL-Hancock half step (Toro, 3rd ed., sec. 14.4) in primitive variables
// for one cell: wh = w - (dt/2) sum_d A_d(w) dw_d / dx_d + (dt/2) S(w), where
// S(w) is gravity on the velocities.  On return dw holds the slopes used
// (all zero after the positivity fallback) and the face states are
// wh -/+ dw_d / 2.  Returns true when the fallback was taken.
template <typename T, int ND, bool HSE>
__device__ __forceinline__ bool hancock(const T (&w)[ND + 2], T (&dw)[ND][ND + 2],
                                        T (&wh)[ND + 2], T hdt, const T (&inv_dx)[3],
                                        T gam, const T (&grav)[3], const CellBG<T> &bg)
{
    constexpr int NV = ND + 2;
    const T rho = HSE ? bg.rho + w[0] : w[0];
    const T pr = HSE ? bg.p + w[NV - 1] : w[NV - 1];
    const T rinv = T(1) / rho;
    T rate[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) rate[q] = T(0);
#pragma unroll
    for (int d = 0; d < ND; ++d) {
        const T un = w[1 + d];
        rate[0] -= (un * dw[d][0] + rho * dw[d][1 + d]) * inv_dx[d];
#pragma unroll
        for (int e = 0; e < ND; ++e) rate[1 + e] -= un * dw[d][1 + e] * inv_dx[d];
        rate[1 + d] -= dw[d][NV - 1] * rinv * inv_dx[d];
        rate[NV - 1] -= (un * dw[d][NV - 1] + gam * pr * dw[d][1 + d]) * inv_dx[d];
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
#pragma unroll
    for (int d = 0; d < ND; ++d) rate[1 + d] += gsrc[d];
#pragma unroll
    for (int q = 0; q < NV; ++q) wh[q] = w[q] + hdt * rate[q];

    // positivity of every predicted face density and pressure
    bool ok = true;
#pragma unroll
    for (int d = 0; d < ND; ++d) {
        T rb_lo = bg.rho, rb_hi = bg.rho, pb_lo = bg.p, pb_hi = bg.p;
        if (HSE && d == 2) { rb_lo = bg.rho_lo; rb_hi = bg.rho_hi; pb_lo = bg.p_lo; pb_hi = bg.p_hi; }
        const T r_lo = rb_lo + (wh[0] - T(0.5) * dw[d][0]);
        const T r_hi = rb_hi + (wh[0] + T(0.5) * dw[d][0]);
        const T p_lo = pb_lo + (wh[NV - 1] - T(0.5) * dw[d][NV - 1]);
        const T p_hi = pb_hi + (wh[NV - 1] + T(0.5) * dw[d][NV - 1]);
        ok = ok && (r_lo > T(0)) && (r_hi > T(0)) && (p_lo > T(0)) && (p_hi > T(0));
    }
    if (!ok) {
#pragma unroll
        for (int d = 0; d < ND; ++d)
#pragma unroll
            for (int q = 0; q < NV; ++q) dw[d][q] = T(0);
#pragma unroll
        for (int q = 0; q < NV; ++q) wh[q] = w[q];
#pragma unroll
        for (int d = 0; d < ND; ++d) wh[1 + d] += hdt * gsrc[d];
    }
    return !ok;
}

// HLLC flux along axis D (Toro, 3rd ed., sec. 10.4-10.6) with Davis wave
// speeds S_L = min(u_L - c_L, u_R - c_R), S_R = max(u_L + c_L, u_R + c_R).
// wl, wr hold (rho', u, p') and (rb, pb) the background at the face; in plain
// mode rb = pb = 0.  The normal momentum flux carries p' (= p in plain mode).
// Branches: 0 <= S_L -> F_L; S_L < 0 <= S* -> F*_L; S* < 0 < S_R -> F*_R;
// S_R <= 0 -> F_R.
template <typename T, int ND, int D, bool HSE>
__device__ __forceinline__ void hllc(const T (&wl)[ND + 2], const T (&wr)[ND + 2], T rb, T pb,
                                     T gam, T (&f)[ND + 2])
{
    constexpr int NV = ND + 2;
    const T rl = HSE ? rb + wl[0] : wl[0];
    const T rr = HSE ? rb + wr[0] : wr[0];
    const T pl = HSE ? pb + wl[NV - 1] : wl[NV - 1];
    const T pr = HSE ? pb + wr[NV - 1] : wr[NV - 1];
    const T ul = wl[1 + D], ur = wr[1 + D];
    const T cl = sqrt(gam * pl / rl);
    const T cr = sqrt(gam * pr / rr);
    const T sl = fmin(ul - cl, ur - cr);
    const T sr = fmax(ul + cl, ur + cr);

    bool left, star;
    T sstar = T(0);
    if (T(0) <= sl) { left = true; star = false; }
    else if (sr <= T(0)) { left = false; star = false; }
    else {
        // pressure difference from the perturbations: the background cancels
        const T dpp = wr[NV - 1] - wl[NV - 1];
        sstar = (dpp + rl * ul * (sl - ul) - rr * ur * (sr - ur)) / (rl * (sl - ul) - rr * (sr - ur));
        left = sstar >= T(0);
        star = true;
    }
    const T rk = left ? rl : rr;
    const T pk = left ? pl : pr;
    const T ppk = left ? wl[NV - 1] : wr[NV - 1];
    const T sk = left ? sl : sr;
    T vk[ND];
#pragma unroll
    for (int e = 0; e < ND; ++e) vk[e] = left ? wl[1 + e] : wr[1 + e];
    const T uk = vk[D];
    T ke = T(0);
#pragma unroll
    for (int e = 0; e < ND; ++e) ke += vk[e] * vk[e];
    const T Ek = pk / (gam - T(1)) + T(0.5) * rk * ke;

    // Euler flux of the chosen side
    const T mflux = rk * uk;
    f[0] = mflux;
#pragma unroll
    for (int e = 0; e < ND; ++e) f[1 + e] = mflux * vk[e];
    f[1 + D] += ppk;
    f[NV - 1] = uk * (Ek + pk);

    if (star) {
        // F*_K = F_K + S_K (U*_K - U_K), U*_K from Toro eq. (10.39)
        const T fac = rk * (sk - uk) / (sk - sstar);
        const T e_star = fac * (Ek / rk + (sstar - uk) * (sstar + pk / (rk * (sk - uk))));
        f[0] += sk * (fac - rk);
#pragma unroll
        for (int e = 0; e < ND; ++e) {
            const T ustar_e = (e == D) ? fac * sstar : fac * vk[e];
            f[1 + e] += sk * (ustar_e - rk * vk[e]);
        }
        f[NV - 1] += sk * (e_star - Ek);
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

// Last-CTA finalisation of a step's time control.  Every CTA calls it once
// with its max signal speed (valid in thread 0) and whether any of its cells
// failed the admissibility check, after storing its part of the new state.
// The CTA that arrives last takes the grid maximum (max is exact, so arrival
// order does not matter), commits the error bits, sets the next dt in FP64
// and advances time.  advance = false only recomputes dt (initialisation).
// Only this CTA writes the fields that every CTA reads at kernel start, and
// it does so after all CTAs have read them.
template <int NT>
__device__ __forceinline__ void finish_step(double smax_cta, bool bad_cta, const StepArgs &a,
                                            int nblocks, double dt_used, bool advance, int *s_last)
{
    if (threadIdx.x == 0) {
        if (bad_cta) atomicOr(&a.ctrl->err_new, 1);
        a.partial[blockIdx.x + (size_t)blockIdx.y * gridDim.x] = smax_cta;
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

}  // namespace hydro
