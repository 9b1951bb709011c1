// ctu2d.cuh -- one step of the corner transport upwind method (Colella
// 1990) for the 2D compressible Euler equations, fused into one kernel.
//
// A CTA owns a TX x TY tile.  In shared memory it
//   1. stages the tile plus a depth-2 halo of U^n as primitives;
//   2. computes, for the tile and a one-cell ring around it (corners
//      included), the one-dimensional MUSCL-Hancock face states of each axis
//      (only that axis's A_d term, half a step of gravity; zero slopes for a
//      cell with a non-positive face density or pressure);
//   3. evaluates first-pass HLLC fluxes at every x face of rows -1..TY and
//      every y face of columns -1..TX;
//   4. corrects the x states of columns -1..TX (tile rows) and the y states
//      of rows -1..TY (tile columns) by -dt/(2 dx_e) times the first-pass flux
//      difference across the other axis, in conserved variables, keeping a
//      cell's uncorrected pair when a corrected density or pressure would not
//      be positive;
//   5. evaluates the final HLLC fluxes of the tile's faces from the corrected
//      states, then applies the MUSCL-Hancock update and sources, stores
//      U^{n+1} and reduces the CFL signal speed.
// Reflecting walls mirror the near-side state on both passes.
#pragma once

#include "hydro_device.cuh"

namespace hydro {

template <typename T, int TX, int TY>
struct Ctu2DSmem {
    static constexpr int NV = 4;
    static constexpr int HX = TX + 4, HY = TY + 4;
    static constexpr int EX = TX + 2, EY = TY + 2;            // tile plus ring
    static constexpr size_t prim = (size_t)NV * HY * HX;
    static constexpr size_t st = (size_t)NV * EY * EX;         // one face-state array
    static constexpr size_t f1x = (size_t)NV * EY * (TX + 1);
    static constexpr size_t f1y = (size_t)NV * (TY + 1) * EX;
    static constexpr size_t fx = (size_t)NV * TY * (TX + 1);
    static constexpr size_t fy = (size_t)NV * (TY + 1) * TX;
    static constexpr size_t elems = prim + 4 * st + f1x + f1y + fx + fy;
    static constexpr size_t bytes = elems * sizeof(T);
    static_assert(bytes <= 226 * 1024, "shared memory of one CTA");
};

// Total primitive (rho, u, v, p) <-> conserved, in the working precision.
template <typename T, int ND>
__device__ __forceinline__ void prim_to_cons_t(const T (&w)[ND + 2], T igm1, T (&u)[ND + 2])
{
    T ke = T(0);
#pragma unroll
    for (int e = 0; e < ND; ++e) {
        u[1 + e] = w[0] * w[1 + e];
        ke += w[1 + e] * w[1 + e];
    }
    u[0] = w[0];
    u[ND + 1] = w[ND + 1] * igm1 + T(0.5) * w[0] * ke;
}

template <typename T, int ND>
__device__ __forceinline__ void cons_to_prim_t(const T (&u)[ND + 2], T gam, T (&w)[ND + 2])
{
    const T rinv = rcp_t(u[0]);
    T m2 = T(0);
#pragma unroll
    for (int e = 0; e < ND; ++e) {
        w[1 + e] = u[1 + e] * rinv;
        m2 += u[1 + e] * u[1 + e];
    }
    w[0] = u[0];
    w[ND + 1] = (gam - T(1)) * (u[ND + 1] - T(0.5) * m2 * rinv);
}

// One-dimensional MUSCL-Hancock predictor along axis d (plain mode): the
// cell state advanced half a step by -A_d(w) dw_d / dx_d and gravity.
template <typename T, int ND>
__device__ __forceinline__ void predict_axis(const T (&w)[ND + 2], const T (&dwd)[ND + 2], int d, T hdt,
                                             T inv_dxd, T gam, const T (&grav)[3], T (&wd)[ND + 2])
{
    constexpr int NV = ND + 2;
    const T rho = w[0], pr = w[NV - 1];
    const T un = w[1 + d];
    const T rinv = rcp_t(rho);
    T r[NV];
    r[0] = -(un * dwd[0] + rho * dwd[1 + d]) * inv_dxd;
#pragma unroll
    for (int e = 0; e < ND; ++e) r[1 + e] = -un * dwd[1 + e] * inv_dxd;
    r[1 + d] -= dwd[NV - 1] * rinv * inv_dxd;
    r[NV - 1] = -(un * dwd[NV - 1] + gam * pr * dwd[1 + d]) * inv_dxd;
#pragma unroll
    for (int e = 0; e < ND; ++e) r[1 + e] += grav[e];
#pragma unroll
    for (int q = 0; q < NV; ++q) wd[q] = w[q] + hdt * r[q];
}

template <typename T, int TX, int TY>
__device__ __forceinline__ void ctu2d_body(const StepArgs &a, int tile, double dtd, unsigned char *smem_raw,
                                           T &smax, bool &bad)
{
    constexpr int ND = 2, NV = 4, NT = TX * TY;
    using S = Ctu2DSmem<T, TX, TY>;
    constexpr int HX = S::HX, HY = S::HY, EX = S::EX, EY = S::EY;
    T *prim = reinterpret_cast<T *>(smem_raw);
    T *sxl = prim + S::prim, *sxh = sxl + S::st, *syl = sxh + S::st, *syh = syl + S::st;
    T *f1x = syh + S::st, *f1y = f1x + S::f1x;
    T *fxs = f1y + S::f1y, *fys = fxs + S::fx;

    const int nx = a.n[0], ny = a.n[1];
    const int tid = threadIdx.x, tx = tid % TX, ty = tid / TX;
    const int x0 = (tile % a.tiles_x) * TX;
    const int y0 = (tile / a.tiles_x) * TY;
    const T *__restrict__ U = static_cast<const T *>(a.U);
    T *__restrict__ Un = static_cast<T *>(a.Unew);
    const long long vs = a.vstride;
    const int gx = x0 + tx, gy = y0 + ty;
    const bool own = gx < nx && gy < ny;
    const T dt = T(dtd), hdt = T(0.5) * T(dtd);
    const T gam = arg_t<T>(a.gamma, a.gamma_f);
    const T igm1 = arg_t<T>(1.0 / (a.gamma - 1.0), a.igm1_f);
    const T inv_dx[3] = {arg_t<T>(a.inv_dx[0], a.inv_dx_f[0]),
                          arg_t<T>(a.inv_dx[1], a.inv_dx_f[1]),
                          T(0)};
    const T grav[3] = {arg_t<T>(a.grav[0], a.grav_f[0]),
                        arg_t<T>(a.grav[1], a.grav_f[1]),
                        T(0)};
    const T hdt_dx[2] = {hdt * inv_dx[0], hdt * inv_dx[1]};   // dt / (2 dx_e)

    auto P = [&](int q, int hy, int hx) -> T & { return prim[(q * HY + hy) * HX + hx]; };
    // face-state arrays over the tile plus ring: cx in [-1, TX], cy in [-1, TY]
    auto SE = [&](T *base, int q, int cy, int cx) -> T & { return base[(q * EY + cy + 1) * EX + cx + 1]; };
    // first-pass x faces fi in [0, TX] (left of column fi), rows cy in [-1, TY];
    // y faces fj in [0, TY], columns cx in [-1, TX]
    auto F1X = [&](int q, int cy, int fi) -> T & { return f1x[(q * EY + cy + 1) * (TX + 1) + fi]; };
    auto F1Y = [&](int q, int fj, int cx) -> T & { return f1y[(q * (TY + 1) + fj) * EX + cx + 1]; };
    auto FX = [&](int q, int cy, int fi) -> T & { return fxs[(q * TY + cy) * (TX + 1) + fi]; };
    auto FY = [&](int q, int fj, int cx) -> T & { return fys[(q * (TY + 1) + fj) * TX + cx]; };

    // ---- 1. the haloed tile as primitives
    for (int i = tid; i < HX * HY; i += NT) {
        const int hx = i % HX, hy = i / HX;
        bool fx, fy;
        const int sx = map_index(x0 + hx - 2, nx, a.bc_lo[0], a.bc_hi[0], fx);
        const int sy = map_index(y0 + hy - 2, ny, a.bc_lo[1], a.bc_hi[1], fy);
        const int c = sy * nx + sx;
        const T r = U[c];
        T m0 = U[c + vs], m1 = U[c + 2 * vs];
        const T e = U[c + 3 * vs];
        if (fx) m0 = -m0;
        if (fy) m1 = -m1;
        const T rinv = rcp_t(r);
        P(0, hy, hx) = r;
        P(1, hy, hx) = m0 * rinv;
        P(2, hy, hx) = m1 * rinv;
        P(3, hy, hx) = (gam - T(1)) * (e - T(0.5) * (m0 * m0 + m1 * m1) * rinv);
    }
    __syncthreads();

    // ---- 2. one-dimensional face states of the tile and its ring
    for (int i = tid; i < EX * EY; i += NT) {
        const int cx = i % EX - 1, cy = i / EX - 1;
        const int hx = cx + 2, hy = cy + 2;
        T w[NV], dw[ND][NV];
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            const T c = P(q, hy, hx);
            w[q] = c;
            dw[0][q] = mc_slope(c - P(q, hy, hx - 1), P(q, hy, hx + 1) - c);
            dw[1][q] = mc_slope(c - P(q, hy - 1, hx), P(q, hy + 1, hx) - c);
        }
        T wd[ND][NV];
        // face densities and pressures {rho_lo, rho_hi, p_lo, p_hi} per axis,
        // formed once for the positivity test and stored as faces
        T rp[ND][4];
        bool ok = true;
#pragma unroll
        for (int d = 0; d < ND; ++d) {
            predict_axis<T, ND>(w, dw[d], d, hdt, inv_dx[d], gam, grav, wd[d]);
            rp[d][0] = wd[d][0] - T(0.5) * dw[d][0];
            rp[d][1] = wd[d][0] + T(0.5) * dw[d][0];
            rp[d][2] = wd[d][NV - 1] - T(0.5) * dw[d][NV - 1];
            rp[d][3] = wd[d][NV - 1] + T(0.5) * dw[d][NV - 1];
            ok = ok && positive(rp[d][0]) && positive(rp[d][1]) && positive(rp[d][2]) && positive(rp[d][3]);
        }
        if (!ok) {
            // zero slopes: every face takes the cell state plus half a step of gravity
#pragma unroll
            for (int d = 0; d < ND; ++d) {
#pragma unroll
                for (int q = 0; q < NV; ++q) {
                    dw[d][q] = T(0);
                    wd[d][q] = w[q] + (q >= 1 && q <= ND ? hdt * grav[q - 1] : T(0));
                }
                rp[d][0] = rp[d][1] = w[0];
                rp[d][2] = rp[d][3] = w[NV - 1];
            }
        }
        auto face = [&](int d, int q, bool hi) -> T {
            if (q == 0) return rp[d][hi ? 1 : 0];
            if (q == NV - 1) return rp[d][hi ? 3 : 2];
            return hi ? wd[d][q] + T(0.5) * dw[d][q] : wd[d][q] - T(0.5) * dw[d][q];
        };
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            SE(sxl, q, cy, cx) = face(0, q, false);
            SE(sxh, q, cy, cx) = face(0, q, true);
            SE(syl, q, cy, cx) = face(1, q, false);
            SE(syh, q, cy, cx) = face(1, q, true);
        }
    }
    __syncthreads();

    // HLLC at the x face left of column fi of row cy (states from sl/sh) or at
    // the y face below row fj of column cx; walls mirror the near side
    auto x_flux = [&](const T *sl, const T *sh, int cy, int fi, T (&f)[NV]) {
        const int gf = x0 + fi;
        const bool w_lo = gf == 0 && a.bc_lo[0] == BC_REFLECT;
        const bool w_hi = gf == nx && a.bc_hi[0] == BC_REFLECT;
        T wl[NV], wr[NV];
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            const T xl = SE(const_cast<T *>(sh), q, cy, fi - 1), xr = SE(const_cast<T *>(sl), q, cy, fi);
            wl[q] = w_lo ? (q == 1 ? -xr : xr) : xl;
            wr[q] = w_hi ? (q == 1 ? -xl : xl) : xr;
        }
        hllc<T, ND, 0, false>(wl, wr, T(0), T(0), gam, igm1, f);
    };
    auto y_flux = [&](const T *sl, const T *sh, int fj, int cx, T (&f)[NV]) {
        const int gf = y0 + fj;
        const bool w_lo = gf == 0 && a.bc_lo[1] == BC_REFLECT;
        const bool w_hi = gf == ny && a.bc_hi[1] == BC_REFLECT;
        T wl[NV], wr[NV];
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            const T yl = SE(const_cast<T *>(sh), q, fj - 1, cx), yr = SE(const_cast<T *>(sl), q, fj, cx);
            wl[q] = w_lo ? (q == 2 ? -yr : yr) : yl;
            wr[q] = w_hi ? (q == 2 ? -yl : yl) : yr;
        }
        hllc<T, ND, 1, false>(wl, wr, T(0), T(0), gam, igm1, f);
    };

    // ---- 3. first-pass fluxes
    for (int i = tid; i < (TX + 1) * EY; i += NT) {
        const int fi = i % (TX + 1), cy = i / (TX + 1) - 1;
        T f[NV];
        x_flux(sxl, sxh, cy, fi, f);
#pragma unroll
        for (int q = 0; q < NV; ++q) F1X(q, cy, fi) = f[q];
    }
    for (int i = tid; i < (TY + 1) * EX; i += NT) {
        const int cx = i % EX - 1, fj = i / EX;
        T f[NV];
        y_flux(syl, syh, fj, cx, f);
#pragma unroll
        for (int q = 0; q < NV; ++q) F1Y(q, fj, cx) = f[q];
    }
    __syncthreads();

    // ---- 4. transverse corrections (both sides of a cell along one axis)
    auto correct = [&](T *lo_arr, T *hi_arr, int cy, int cx, const T (&df)[NV], T k) {
        T wc[2][NV];
        bool ok = true;
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            T w[NV], u[NV];
#pragma unroll
            for (int q = 0; q < NV; ++q) w[q] = SE(s ? hi_arr : lo_arr, q, cy, cx);
            prim_to_cons_t<T, ND>(w, igm1, u);
#pragma unroll
            for (int q = 0; q < NV; ++q) u[q] -= k * df[q];
            cons_to_prim_t<T, ND>(u, gam, wc[s]);
            ok = ok && positive(wc[s][0]) && positive(wc[s][NV - 1]);
        }
        if (ok) {
#pragma unroll
            for (int s = 0; s < 2; ++s)
#pragma unroll
                for (int q = 0; q < NV; ++q) SE(s ? hi_arr : lo_arr, q, cy, cx) = wc[s][q];
        }
    };
    for (int i = tid; i < EX * TY; i += NT) {          // x states: columns -1..TX, tile rows
        const int cx = i % EX - 1, cy = i / EX;
        T df[NV];
#pragma unroll
        for (int q = 0; q < NV; ++q) df[q] = F1Y(q, cy + 1, cx) - F1Y(q, cy, cx);
        correct(sxl, sxh, cy, cx, df, hdt_dx[1]);
    }
    for (int i = tid; i < TX * EY; i += NT) {          // y states: tile columns, rows -1..TY
        const int cx = i % TX, cy = i / TX - 1;
        T df[NV];
#pragma unroll
        for (int q = 0; q < NV; ++q) df[q] = F1X(q, cy, cx + 1) - F1X(q, cy, cx);
        correct(syl, syh, cy, cx, df, hdt_dx[0]);
    }
    __syncthreads();

    // ---- 5. final fluxes of the tile's faces
    for (int i = tid; i < (TX + 1) * TY; i += NT) {
        const int fi = i % (TX + 1), cy = i / (TX + 1);
        T f[NV];
        x_flux(sxl, sxh, cy, fi, f);
#pragma unroll
        for (int q = 0; q < NV; ++q) FX(q, cy, fi) = f[q];
    }
    for (int i = tid; i < (TY + 1) * TX; i += NT) {
        const int cx = i % TX, fj = i / TX;
        T f[NV];
        y_flux(syl, syh, fj, cx, f);
#pragma unroll
        for (int q = 0; q < NV; ++q) FY(q, fj, cx) = f[q];
    }
    __syncthreads();

    // ---- update (MUSCL-Hancock sources), admissibility, CFL signal speed
    smax = T(0);
    bad = false;
    if (own) {
        const int c = gy * nx + gx;
        T u[NV], du[NV];
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            u[q] = U[c + q * vs];
            du[q] = -((FX(q, ty, tx + 1) - FX(q, ty, tx)) * inv_dx[0]
                      + (FY(q, ty + 1, tx) - FY(q, ty, tx)) * inv_dx[1]);
        }
        const T msrc = grav[0] * T(0.5) * (FX(0, ty, tx) + FX(0, ty, tx + 1))
                     + grav[1] * T(0.5) * (FY(0, ty, tx) + FY(0, ty + 1, tx));
        const T r_old = u[0];
        const T r_new = r_old + dt * du[0];
        u[0] = r_new;
        const T rsum = T(0.5) * (r_old + r_new);
        u[1] += dt * (du[1] + grav[0] * rsum);
        u[2] += dt * (du[2] + grav[1] * rsum);
        u[3] += dt * (du[3] + msrc);
#pragma unroll
        for (int q = 0; q < NV; ++q) Un[c + q * vs] = u[q];
        const T rinv = rcp_t(u[0]);
        const T pres = (gam - T(1)) * (u[3] - half_nonneg(u[1] * u[1] + u[2] * u[2]) * rinv);
        const T gp = gam * pres;
        const T cs = gp * rsqrt_t(gp * u[0]);
        const T s = signal_speed<T, 2>(u + 1, rinv, cs, inv_dx);
        if (!(u[0] > T(0)) || !(pres > T(0)) || !isfinite(s)) bad = true;
        else smax = s;
    }
}

template <typename T, int TX, int TY>
__global__ void __launch_bounds__(TX * TY) ctu2d_kernel(const StepArgs a)
{
    constexpr int NT = TX * TY;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[32];
    __shared__ int s_last;
    const double t_now = a.ctrl->t;
    const double dt_cfl = a.ctrl->dt_next;
    // frozen: nothing moves (the host finds the current buffer from the step count)
    if (t_now >= a.t_end || a.ctrl->err != 0 || a.ctrl->step >= a.step_end) return;
    const double dtd = (dt_cfl >= a.t_end - t_now) ? a.t_end - t_now : dt_cfl;
    T smax;
    bool bad;
    ctu2d_body<T, TX, TY>(a, blockIdx.x, dtd, smem_raw, smax, bad);
    const bool bad_cta = __syncthreads_or(bad) != 0;
    const double m = block_max_t<NT, T>(smax, red);
    finish_step<NT>(m, bad_cta, a, gridDim.x * gridDim.y, blockIdx.x + blockIdx.y * gridDim.x, dtd, true,
                    &s_last);
}

}  // namespace hydro
