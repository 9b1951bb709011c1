// pair_math.cuh -- FP32 arithmetic of the update on pairs of cells.
//
// The paired FP32 step kernel gives each thread two x-adjacent cells and
// evaluates their slopes, half steps, HLLC fluxes and updates together:
// additions, multiplications and fused multiply-adds act on both cells at
// once as packed f32x2 operations (one instruction for two independent
// results, each rounded exactly as the scalar operation), while square-root
// reciprocals, reciprocals, minima, maxima, comparisons and selects stay
// per lane.  The two lanes never interact, so a cell's result does not
// depend on which cell shares its pair: a lone cell (the tile's ring, the
// high-side faces) is evaluated as a pair with itself and gets the bits it
// would get in any other pair.
//
// The formulas are those of hydro_device.cuh (MC limiter, MUSCL-Hancock half
// step with the positivity fallback, HLLC with Davis wave speeds, the
// conservative update with the gravity sources); only the grouping of the
// operations into packed instructions is new.
#pragma once

#include <cuda_runtime.h>

#include "hydro_device.cuh"

namespace hydro {

using f2 = float2;

__device__ __forceinline__ f2 pr(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ f2 bc(float s) { return make_float2(s, s); }
__device__ __forceinline__ f2 add2(f2 a, f2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ f2 mul2(f2 a, f2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) { return __ffma2_rn(a, b, c); }
// a - b as a + (-1) b: one rounding, the same value as the subtraction
__device__ __forceinline__ f2 sub2(f2 a, f2 b) { return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a); }

// per-lane operations
__device__ __forceinline__ f2 rcp2(f2 a) { return pr(__fdividef(1.0f, a.x), __fdividef(1.0f, a.y)); }
__device__ __forceinline__ f2 rsqrt2(f2 a) { return pr(rsqrtf(a.x), rsqrtf(a.y)); }
__device__ __forceinline__ f2 min2(f2 a, f2 b) { return pr(fminf(a.x, b.x), fminf(a.y, b.y)); }
__device__ __forceinline__ f2 max2(f2 a, f2 b) { return pr(fmaxf(a.x, b.x), fmaxf(a.y, b.y)); }
__device__ __forceinline__ f2 abs2(f2 a) { return pr(fabsf(a.x), fabsf(a.y)); }

struct b2 {
    bool x, y;
};
__device__ __forceinline__ f2 sel2(b2 m, f2 a, f2 b) { return pr(m.x ? a.x : b.x, m.y ? a.y : b.y); }

// MC-limited slope of each lane: sign(dr) min(2|dl|, 2|dr|, |dl+dr|/2) when
// dl dr > 0, else 0.
__device__ __forceinline__ f2 mc_slope2(f2 dl, f2 dr)
{
    const f2 m = min2(abs2(dl), abs2(dr));
    const f2 twice = add2(m, m);
    const f2 half = mul2(abs2(add2(dl, dr)), bc(0.5f));
    const f2 a = min2(twice, half);
    const f2 p = mul2(dl, dr);
    return pr(p.x > 0.0f ? copysignf(a.x, dr.x) : 0.0f, p.y > 0.0f ? copysignf(a.y, dr.y) : 0.0f);
}

// Background of the plane both cells of a pair share (x-pairs lie in one
// z plane): scalars, all zero in plain mode.
template <bool HSE>
__device__ __forceinline__ CellBG<float> plane_bg(const PlaneBGT<float> *bg, int k)
{
    return cell_bg<float, HSE>(bg, k);
}

// MUSCL-Hancock half step (Toro, 3rd ed., sec. 14.4) of a pair of cells in
// primitive variables with the per-lane positivity fallback: a lane whose
// predicted face density or pressure along any axis is not positive gets
// zero slopes and wh = w + (dt/2) (gravity source).  gz: gravity along z
// only.  On return dw holds the slopes used.
template <bool HSE, bool GZ>
__device__ __forceinline__ void hancock2(const f2 (&w)[5], f2 (&dw)[3][5], f2 (&wh)[5], float hdt,
                                         const float (&inv_dx)[3], float gam, const float (&grav)[3],
                                         const CellBG<float> &bg)
{
    const f2 rho = HSE ? add2(bc(bg.rho), w[0]) : w[0];
    const f2 pres = HSE ? add2(bc(bg.p), w[4]) : w[4];
    const f2 rinv = rcp2(rho);
    const f2 gp = mul2(bc(gam), pres);
    f2 rate[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) rate[q] = bc(0.0f);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const f2 nun = mul2(w[1 + d], bc(-inv_dx[d]));           // -u_d / dx_d
        const f2 nrho = mul2(bc(-inv_dx[d]), rho);
        const f2 nrinv = mul2(bc(-inv_dx[d]), rinv);
        const f2 ngp = mul2(bc(-inv_dx[d]), gp);
        rate[0] = fma2(nun, dw[d][0], rate[0]);
        rate[0] = fma2(nrho, dw[d][1 + d], rate[0]);
#pragma unroll
        for (int e = 0; e < 3; ++e) rate[1 + e] = fma2(nun, dw[d][1 + e], rate[1 + e]);
        rate[1 + d] = fma2(nrinv, dw[d][4], rate[1 + d]);
        rate[4] = fma2(nun, dw[d][4], rate[4]);
        rate[4] = fma2(ngp, dw[d][1 + d], rate[4]);
    }
    // gravity on the velocities: g rho'/rho - B/rho in HSE mode, g otherwise
    f2 gsrc[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) gsrc[d] = HSE ? mul2(bc(grav[d]), mul2(w[0], rinv)) : bc(grav[d]);
    if constexpr (HSE) {
        const f2 wz = w[3];
        rate[0] = fma2(mul2(wz, bc(-inv_dx[2])), bc(bg.drho), rate[0]);
        rate[4] = fma2(mul2(wz, bc(-inv_dx[2])), bc(bg.dp), rate[4]);
        gsrc[2] = fma2(bc(-bg.B), rinv, gsrc[2]);
    }
#pragma unroll
    for (int d = 0; d < 3; ++d)
        if (!GZ || d == 2) rate[1 + d] = add2(rate[1 + d], gsrc[d]);
    const f2 h = bc(hdt);
#pragma unroll
    for (int q = 0; q < 5; ++q) wh[q] = fma2(h, rate[q], w[q]);

    // positivity of every predicted face density and pressure, per lane
    bool okx = true, oky = true;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        float rb_lo = bg.rho, rb_hi = bg.rho, pb_lo = bg.p, pb_hi = bg.p;
        if (HSE && d == 2) { rb_lo = bg.rho_lo; rb_hi = bg.rho_hi; pb_lo = bg.p_lo; pb_hi = bg.p_hi; }
        const f2 hr = mul2(bc(0.5f), dw[d][0]);
        const f2 hp = mul2(bc(0.5f), dw[d][4]);
        // (plain mode: no addition of the zero background)
        const f2 r_lo = HSE ? add2(bc(rb_lo), sub2(wh[0], hr)) : sub2(wh[0], hr);
        const f2 r_hi = HSE ? add2(bc(rb_hi), add2(wh[0], hr)) : add2(wh[0], hr);
        const f2 p_lo = HSE ? add2(bc(pb_lo), sub2(wh[4], hp)) : sub2(wh[4], hp);
        const f2 p_hi = HSE ? add2(bc(pb_hi), add2(wh[4], hp)) : add2(wh[4], hp);
        okx = okx && r_lo.x > 0.0f && r_hi.x > 0.0f && p_lo.x > 0.0f && p_hi.x > 0.0f;
        oky = oky && r_lo.y > 0.0f && r_hi.y > 0.0f && p_lo.y > 0.0f && p_hi.y > 0.0f;
    }
    if (!okx || !oky) {
        const b2 keep{okx, oky};
#pragma unroll
        for (int d = 0; d < 3; ++d)
#pragma unroll
            for (int q = 0; q < 5; ++q) dw[d][q] = sel2(keep, dw[d][q], bc(0.0f));
        f2 w0[5];
#pragma unroll
        for (int q = 0; q < 5; ++q) w0[q] = w[q];
#pragma unroll
        for (int d = 0; d < 3; ++d)
            if (!GZ || d == 2) w0[1 + d] = fma2(h, gsrc[d], w0[1 + d]);
#pragma unroll
        for (int q = 0; q < 5; ++q) wh[q] = sel2(keep, wh[q], w0[q]);
    }
}

// HLLC flux along axis D (Toro, 3rd ed., sec. 10.4-10.6) of a pair of
// faces, Davis wave speeds, branch tie S* = 0 to the left; (rb, pb) the
// background at the faces (zero in plain mode), the normal momentum flux
// carries p'.  The star correction is formed through the factor
// h = S_K (S* - u_K) / (S_K - S*) as in hllc() of hydro_device.cuh, and the
// fan's branch is applied by per-lane selects.
template <int D, bool HSE>
__device__ __forceinline__ void hllc2(const f2 (&wl)[5], const f2 (&wr)[5], float rb, float pb, float gam,
                                      float igm1, f2 (&f)[5])
{
    const f2 rl = HSE ? add2(bc(rb), wl[0]) : wl[0];
    const f2 rr = HSE ? add2(bc(rb), wr[0]) : wr[0];
    const f2 pl = HSE ? add2(bc(pb), wl[4]) : wl[4];
    const f2 prr = HSE ? add2(bc(pb), wr[4]) : wr[4];
    const f2 ul = wl[1 + D], ur = wr[1 + D];
    const f2 gpl = mul2(bc(gam), pl), gpr = mul2(bc(gam), prr);
    const f2 cl = mul2(gpl, rsqrt2(mul2(gpl, rl)));
    const f2 cr = mul2(gpr, rsqrt2(mul2(gpr, rr)));
    const f2 sl = min2(sub2(ul, cl), sub2(ur, cr));
    const f2 sr = max2(add2(ul, cl), add2(ur, cr));
    const f2 dpp = sub2(wr[4], wl[4]);                 // background cancels in the difference
    const f2 ml = mul2(rl, sub2(sl, ul)), mr = mul2(rr, sub2(sr, ur));
    const f2 num = sub2(fma2(ml, ul, dpp), mul2(mr, ur));
    const f2 den = sub2(ml, mr);
    const f2 sstar = pr(__fdividef(num.x, den.x), __fdividef(num.y, den.y));
    b2 left, star;
    {
        const bool supl_x = sl.x >= 0.0f, supl_y = sl.y >= 0.0f;
        const bool supr_x = sr.x <= 0.0f, supr_y = sr.y <= 0.0f;
        left = b2{supl_x || (!supr_x && sstar.x >= 0.0f), supl_y || (!supr_y && sstar.y >= 0.0f)};
        star = b2{!supl_x && !supr_x, !supl_y && !supr_y};
    }
    const f2 rk = sel2(left, rl, rr);
    const f2 pk = sel2(left, pl, prr);
    const f2 ppk = sel2(left, wl[4], wr[4]);
    const f2 sk = sel2(left, sl, sr);
    const f2 mk = sel2(left, ml, mr);
    f2 vk[3];
#pragma unroll
    for (int e = 0; e < 3; ++e) vk[e] = sel2(left, wl[1 + e], wr[1 + e]);
    const f2 uk = vk[D];
    const f2 ke = fma2(vk[2], vk[2], fma2(vk[1], vk[1], mul2(vk[0], vk[0])));
    // E_K + p_K = p_K gamma / (gamma - 1) + rho_K |v_K|^2 / 2
    const f2 hk = fma2(pk, bc(igm1 + 1.0f), mul2(mul2(bc(0.5f), rk), ke));

    // Euler flux of the chosen side
    const f2 mflux = mul2(rk, uk);
    f[0] = mflux;
#pragma unroll
    for (int e = 0; e < 3; ++e) f[1 + e] = mul2(mflux, vk[e]);
    f[1 + D] = add2(f[1 + D], ppk);
    f[4] = mul2(uk, hk);

    // F*_K = F_K + S_K (U*_K - U_K), applied only inside the fan
    const f2 h = mul2(mul2(sk, rcp2(sub2(sk, sstar))), sub2(sstar, uk));
    const f2 c0 = mul2(rk, h);                         // S_K (rho*_K - rho_K)
    f[0] = sel2(star, add2(f[0], c0), f[0]);
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        const f2 fs = fma2(c0, (e == D) ? sk : vk[e], f[1 + e]);
        f[1 + e] = sel2(star, fs, f[1 + e]);
    }
    f[4] = sel2(star, fma2(h, fma2(mk, sstar, hk), f[4]), f[4]);
}

}  // namespace hydro
