// ctu3d.cuh -- one step of the corner transport upwind method (Colella
// 1990) for the 3D compressible Euler equations, fused into one kernel.
//
// A CTA owns a TX x TY x TZ block of cells (the transverse corrections of a
// face state need first-pass fluxes one cell beyond the block in every
// direction, so the block is staged whole rather than marched in z).  In
// shared memory it
//   1. stages the block plus a depth-2 halo of U^n as primitives;
//   2. computes the one-dimensional MUSCL-Hancock face states of each axis
//      (that axis's A_d term and half a step of gravity; zero slopes for a
//      cell with a non-positive face density or pressure) for the block and
//      a one-cell shell around it;
//   3. evaluates first-pass HLLC fluxes through every face of the shell;
//   4. corrects each axis's face states of the cells that border a block
//      face along that axis by -dt/(2 dx_e) times the first-pass flux
//      differences of the two other axes, in conserved variables (a cell
//      keeps its uncorrected pair when a corrected density or pressure would
//      not be positive);
//   5. evaluates the final HLLC fluxes through the block's faces from the
//      corrected states (into the first-pass arrays), then applies the
//      MUSCL-Hancock update and sources, stores U^{n+1} and reduces the CFL
//      signal speed.
// Reflecting walls mirror the near-side state on both passes.
#pragma once

#include <type_traits>

#include "ctu2d.cuh"   // prim_to_cons_t, cons_to_prim_t, predict_axis

namespace hydro {

template <typename T, int TX, int TY, int TZ>
struct Ctu3DSmem {
    static constexpr int NV = 5;
    static constexpr int HX = TX + 4, HY = TY + 4, HZ = TZ + 4;
    static constexpr int EX = TX + 2, EY = TY + 2, EZ = TZ + 2;   // block plus shell
    static constexpr size_t prim = (size_t)NV * HZ * HY * HX;
    static constexpr size_t st = (size_t)NV * EZ * EY * EX;        // one face-state array
    static constexpr size_t f1x = (size_t)NV * EZ * EY * (TX + 1);
    static constexpr size_t f1y = (size_t)NV * EZ * (TY + 1) * EX;
    static constexpr size_t f1z = (size_t)NV * (TZ + 1) * EY * EX;
    static constexpr size_t elems = prim + 6 * st + f1x + f1y + f1z;
    static constexpr size_t bytes = elems * sizeof(T);
    static_assert(bytes <= 226 * 1024, "shared memory of one CTA");
};

template <typename T, int TX, int TY, int TZ>
__device__ __forceinline__ void ctu3d_body(const StepArgs &a, int block, double dtd, unsigned char *smem_raw,
                                           T &smax, bool &bad)
{
    constexpr int ND = 3, NV = 5, NT = TX * TY * TZ;
    using S = Ctu3DSmem<T, TX, TY, TZ>;
    constexpr int HX = S::HX, HY = S::HY, HZ = S::HZ, EX = S::EX, EY = S::EY, EZ = S::EZ;
    T *prim = reinterpret_cast<T *>(smem_raw);
    T *sl[3], *sh[3];
    sl[0] = prim + S::prim;
    sh[0] = sl[0] + S::st;
    sl[1] = sh[0] + S::st;
    sh[1] = sl[1] + S::st;
    sl[2] = sh[1] + S::st;
    sh[2] = sl[2] + S::st;
    T *f1x = sh[2] + S::st, *f1y = f1x + S::f1x, *f1z = f1y + S::f1y;

    const int nx = a.n[0], ny = a.n[1], nz = a.n[2];
    const int bx_n = (nx + TX - 1) / TX, by_n = (ny + TY - 1) / TY;
    const int x0 = (block % bx_n) * TX;
    const int y0 = ((block / bx_n) % by_n) * TY;
    const int z0 = (block / (bx_n * by_n)) * TZ;
    const int tid = threadIdx.x, tx = tid % TX, ty = (tid / TX) % TY, tz = tid / (TX * TY);
    const T *__restrict__ U = static_cast<const T *>(a.U);
    T *__restrict__ Un = static_cast<T *>(a.Unew);
    const long long vs = a.vstride;
    const int plane = static_cast<int>(a.plane);
    const int gx = x0 + tx, gy = y0 + ty, gz = z0 + tz;
    const bool own = gx < nx && gy < ny && gz < nz;
    const T dt = T(dtd), hdt = T(0.5) * T(dtd);
    const T gam = T(a.gamma);
    const T igm1 = T(1.0 / (a.gamma - 1.0));
    const T inv_dx[3] = {T(a.inv_dx[0]), T(a.inv_dx[1]), T(a.inv_dx[2])};
    const T grav[3] = {T(a.grav[0]), T(a.grav[1]), T(a.grav[2])};
    const T hdt_dx[3] = {hdt * inv_dx[0], hdt * inv_dx[1], hdt * inv_dx[2]};   // dt / (2 dx_e)
    const int n3[3] = {nx, ny, nz}, o3[3] = {x0, y0, z0};

    auto P = [&](int q, int hz, int hy, int hx) -> T & { return prim[((q * HZ + hz) * HY + hy) * HX + hx]; };
    // face states over the block plus shell: c in [-1, T]
    auto SE = [&](T *base, int q, int cz, int cy, int cx) -> T & {
        return base[((q * EZ + cz + 1) * EY + cy + 1) * EX + cx + 1];
    };
    // flux through the low face of cell f along the array's axis (f in [0, T]),
    // the other two coordinates in [-1, T]
    auto FXA = [&](int q, int cz, int cy, int fi) -> T & {
        return f1x[((q * EZ + cz + 1) * EY + cy + 1) * (TX + 1) + fi];
    };
    auto FYA = [&](int q, int cz, int fj, int cx) -> T & {
        return f1y[((q * EZ + cz + 1) * (TY + 1) + fj) * EX + cx + 1];
    };
    auto FZA = [&](int q, int fk, int cy, int cx) -> T & {
        return f1z[((q * (TZ + 1) + fk) * EY + cy + 1) * EX + cx + 1];
    };

    // ---- 1. the haloed block as primitives
    for (int i = tid; i < HX * HY * HZ; i += NT) {
        const int hx = i % HX, hy = (i / HX) % HY, hz = i / (HX * HY);
        bool fx, fy, fz;
        const int sx = map_index(x0 + hx - 2, nx, a.bc_lo[0], a.bc_hi[0], fx);
        const int sy = map_index(y0 + hy - 2, ny, a.bc_lo[1], a.bc_hi[1], fy);
        const int sz = map_index(z0 + hz - 2, nz, a.bc_lo[2], a.bc_hi[2], fz);
        const long long c = (long long)sz * plane + sy * nx + sx;
        const T r = U[c];
        T m0 = U[c + vs], m1 = U[c + 2 * vs], m2 = U[c + 3 * vs];
        const T e = U[c + 4 * vs];
        if (fx) m0 = -m0;
        if (fy) m1 = -m1;
        if (fz) m2 = -m2;
        const T rinv = rcp_t(r);
        P(0, hz, hy, hx) = r;
        P(1, hz, hy, hx) = m0 * rinv;
        P(2, hz, hy, hx) = m1 * rinv;
        P(3, hz, hy, hx) = m2 * rinv;
        P(4, hz, hy, hx) = (gam - T(1)) * (e - T(0.5) * (m0 * m0 + m1 * m1 + m2 * m2) * rinv);
    }
    __syncthreads();

    // ---- 2. one-dimensional face states of the block and its shell
    for (int i = tid; i < EX * EY * EZ; i += NT) {
        const int cx = i % EX - 1, cy = (i / EX) % EY - 1, cz = i / (EX * EY) - 1;
        const int hx = cx + 2, hy = cy + 2, hz = cz + 2;
        T w[NV], dw[ND][NV];
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            const T c = P(q, hz, hy, hx);
            w[q] = c;
            dw[0][q] = mc_slope(c - P(q, hz, hy, hx - 1), P(q, hz, hy, hx + 1) - c);
            dw[1][q] = mc_slope(c - P(q, hz, hy - 1, hx), P(q, hz, hy + 1, hx) - c);
            dw[2][q] = mc_slope(c - P(q, hz - 1, hy, hx), P(q, hz + 1, hy, hx) - c);
        }
        T wd[ND][NV];
        bool ok = true;
#pragma unroll
        for (int d = 0; d < ND; ++d) {
            predict_axis<T, ND>(w, dw[d], d, hdt, inv_dx[d], gam, grav, wd[d]);
            ok = ok && positive(wd[d][0] - T(0.5) * dw[d][0]) && positive(wd[d][0] + T(0.5) * dw[d][0])
                    && positive(wd[d][NV - 1] - T(0.5) * dw[d][NV - 1])
                    && positive(wd[d][NV - 1] + T(0.5) * dw[d][NV - 1]);
        }
        if (!ok) {
#pragma unroll
            for (int d = 0; d < ND; ++d)
#pragma unroll
                for (int q = 0; q < NV; ++q) {
                    dw[d][q] = T(0);
                    wd[d][q] = w[q] + (q >= 1 && q <= ND ? hdt * grav[q - 1] : T(0));
                }
        }
#pragma unroll
        for (int d = 0; d < ND; ++d)
#pragma unroll
            for (int q = 0; q < NV; ++q) {
                SE(sl[d], q, cz, cy, cx) = wd[d][q] - T(0.5) * dw[d][q];
                SE(sh[d], q, cz, cy, cx) = wd[d][q] + T(0.5) * dw[d][q];
            }
    }
    __syncthreads();

    // HLLC through the low face of cell c along axis D (states of c - e_D
    // and c); walls mirror the near side
    auto face_flux = [&](auto DC, int cz, int cy, int cx, T (&f)[NV]) {
        constexpr int D = decltype(DC)::value;
        const int cc[3] = {cx, cy, cz};
        const int gf = o3[D] + cc[D];
        const bool w_lo = gf == 0 && a.bc_lo[D] == BC_REFLECT;
        const bool w_hi = gf == n3[D] && a.bc_hi[D] == BC_REFLECT;
        const int lx = cx - (D == 0), ly = cy - (D == 1), lz = cz - (D == 2);
        T wl[NV], wr[NV];
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            const T vl = SE(sh[D], q, lz, ly, lx), vr = SE(sl[D], q, cz, cy, cx);
            wl[q] = w_lo ? (q == 1 + D ? -vr : vr) : vl;
            wr[q] = w_hi ? (q == 1 + D ? -vl : vl) : vr;
        }
        hllc<T, ND, D, false>(wl, wr, T(0), T(0), gam, igm1, f);
    };
    using D0 = std::integral_constant<int, 0>;
    using D1 = std::integral_constant<int, 1>;
    using D2 = std::integral_constant<int, 2>;

    // ---- 3. first-pass fluxes through every face of the shell
    for (int i = tid; i < (TX + 1) * EY * EZ; i += NT) {
        const int fi = i % (TX + 1), cy = (i / (TX + 1)) % EY - 1, cz = i / ((TX + 1) * EY) - 1;
        T f[NV];
        face_flux(D0{}, cz, cy, fi, f);
#pragma unroll
        for (int q = 0; q < NV; ++q) FXA(q, cz, cy, fi) = f[q];
    }
    for (int i = tid; i < EX * (TY + 1) * EZ; i += NT) {
        const int cx = i % EX - 1, fj = (i / EX) % (TY + 1), cz = i / (EX * (TY + 1)) - 1;
        T f[NV];
        face_flux(D1{}, cz, fj, cx, f);
#pragma unroll
        for (int q = 0; q < NV; ++q) FYA(q, cz, fj, cx) = f[q];
    }
    for (int i = tid; i < EX * EY * (TZ + 1); i += NT) {
        const int cx = i % EX - 1, cy = (i / EX) % EY - 1, fk = i / (EX * EY);
        T f[NV];
        face_flux(D2{}, fk, cy, cx, f);
#pragma unroll
        for (int q = 0; q < NV; ++q) FZA(q, fk, cy, cx) = f[q];
    }
    __syncthreads();

    // ---- 4. transverse corrections of both face states of a cell along d
    auto correct = [&](int d, int cz, int cy, int cx) {
        T df[2][NV];
        T k[2];
        int m = 0;
#pragma unroll
        for (int e = 0; e < ND; ++e) {
            if (e == d) continue;
#pragma unroll
            for (int q = 0; q < NV; ++q)
                df[m][q] = e == 0 ? FXA(q, cz, cy, cx + 1) - FXA(q, cz, cy, cx)
                         : e == 1 ? FYA(q, cz, cy + 1, cx) - FYA(q, cz, cy, cx)
                                  : FZA(q, cz + 1, cy, cx) - FZA(q, cz, cy, cx);
            k[m] = hdt_dx[e];
            ++m;
        }
        T wc[2][NV];
        bool ok = true;
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            T w[NV], u[NV];
#pragma unroll
            for (int q = 0; q < NV; ++q) w[q] = SE(s ? sh[d] : sl[d], q, cz, cy, cx);
            prim_to_cons_t<T, ND>(w, igm1, u);
#pragma unroll
            for (int j = 0; j < 2; ++j)
#pragma unroll
                for (int q = 0; q < NV; ++q) u[q] -= k[j] * df[j][q];
            cons_to_prim_t<T, ND>(u, gam, wc[s]);
            ok = ok && positive(wc[s][0]) && positive(wc[s][NV - 1]);
        }
        if (ok) {
#pragma unroll
            for (int s = 0; s < 2; ++s)
#pragma unroll
                for (int q = 0; q < NV; ++q) SE(s ? sh[d] : sl[d], q, cz, cy, cx) = wc[s][q];
        }
    };
    for (int i = tid; i < EX * TY * TZ; i += NT)   // x states: x in [-1, TX], block y and z
        correct(0, i / (EX * TY), (i / EX) % TY, i % EX - 1);
    for (int i = tid; i < TX * EY * TZ; i += NT)   // y states
        correct(1, i / (TX * EY), (i / TX) % EY - 1, i % TX);
    for (int i = tid; i < TX * TY * EZ; i += NT)   // z states
        correct(2, i / (TX * TY) - 1, (i / TX) % TY, i % TX);
    __syncthreads();

    // ---- 5. final fluxes through the block's faces (into the first-pass arrays)
    for (int i = tid; i < (TX + 1) * TY * TZ; i += NT) {
        const int fi = i % (TX + 1), cy = (i / (TX + 1)) % TY, cz = i / ((TX + 1) * TY);
        T f[NV];
        face_flux(D0{}, cz, cy, fi, f);
#pragma unroll
        for (int q = 0; q < NV; ++q) FXA(q, cz, cy, fi) = f[q];
    }
    for (int i = tid; i < TX * (TY + 1) * TZ; i += NT) {
        const int cx = i % TX, fj = (i / TX) % (TY + 1), cz = i / (TX * (TY + 1));
        T f[NV];
        face_flux(D1{}, cz, fj, cx, f);
#pragma unroll
        for (int q = 0; q < NV; ++q) FYA(q, cz, fj, cx) = f[q];
    }
    for (int i = tid; i < TX * TY * (TZ + 1); i += NT) {
        const int cx = i % TX, cy = (i / TX) % TY, fk = i / (TX * TY);
        T f[NV];
        face_flux(D2{}, fk, cy, cx, f);
#pragma unroll
        for (int q = 0; q < NV; ++q) FZA(q, fk, cy, cx) = f[q];
    }
    __syncthreads();

    // ---- update (MUSCL-Hancock sources), admissibility, CFL signal speed
    smax = T(0);
    bad = false;
    if (own) {
        const long long c = (long long)gz * plane + gy * nx + gx;
        T u[NV], du[NV];
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            u[q] = U[c + q * vs];
            du[q] = -((FXA(q, tz, ty, tx + 1) - FXA(q, tz, ty, tx)) * inv_dx[0]
                      + (FYA(q, tz, ty + 1, tx) - FYA(q, tz, ty, tx)) * inv_dx[1]
                      + (FZA(q, tz + 1, ty, tx) - FZA(q, tz, ty, tx)) * inv_dx[2]);
        }
        const T msrc = grav[0] * T(0.5) * (FXA(0, tz, ty, tx) + FXA(0, tz, ty, tx + 1))
                     + grav[1] * T(0.5) * (FYA(0, tz, ty, tx) + FYA(0, tz, ty + 1, tx))
                     + grav[2] * T(0.5) * (FZA(0, tz, ty, tx) + FZA(0, tz + 1, ty, tx));
        const T r_old = u[0];
        const T r_new = r_old + dt * du[0];
        u[0] = r_new;
        const T rsum = T(0.5) * (r_old + r_new);
#pragma unroll
        for (int d = 0; d < ND; ++d) u[1 + d] += dt * (du[1 + d] + grav[d] * rsum);
        u[4] += dt * (du[4] + msrc);
#pragma unroll
        for (int q = 0; q < NV; ++q) Un[c + q * vs] = u[q];
        const T rinv = rcp_t(u[0]);
        const T vx = u[1] * rinv, vy = u[2] * rinv, vz = u[3] * rinv;
        const T pres = (gam - T(1)) * (u[4] - T(0.5) * (u[1] * u[1] + u[2] * u[2] + u[3] * u[3]) * rinv);
        const T gp = gam * pres;
        const T cs = gp * rsqrt_t(gp * u[0]);
        const T s = (fabs(vx) + cs) * inv_dx[0] + (fabs(vy) + cs) * inv_dx[1] + (fabs(vz) + cs) * inv_dx[2];
        if (!(u[0] > T(0)) || !(pres > T(0)) || !isfinite(s)) bad = true;
        else smax = s;
    }
}

template <typename T, int TX, int TY, int TZ>
__global__ void __launch_bounds__(TX * TY * TZ) ctu3d_kernel(const StepArgs a)
{
    constexpr int NT = TX * TY * TZ;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[32];
    __shared__ int s_last;
    const double t_now = a.ctrl->t;
    const double dt_cfl = a.ctrl->dt_next;
    if (t_now >= a.t_end || a.ctrl->err != 0 || a.ctrl->step >= a.step_end) {
        // U^n carried over
        constexpr int NV = 5;
        const int nx = a.n[0], ny = a.n[1];
        const int bx_n = (nx + TX - 1) / TX, by_n = (ny + TY - 1) / TY;
        const int gx = (blockIdx.x % bx_n) * TX + threadIdx.x % TX;
        const int gy = ((blockIdx.x / bx_n) % by_n) * TY + (threadIdx.x / TX) % TY;
        const int gz = (blockIdx.x / (bx_n * by_n)) * TZ + threadIdx.x / (TX * TY);
        if (gx < nx && gy < ny && gz < a.n[2])
            for (int q = 0; q < NV; ++q) {
                const long long c = q * a.vstride + (long long)gz * a.plane + (long long)gy * nx + gx;
                static_cast<T *>(a.Unew)[c] = static_cast<const T *>(a.U)[c];
            }
        return;
    }
    const double dtd = (dt_cfl >= a.t_end - t_now) ? a.t_end - t_now : dt_cfl;
    T smax;
    bool bad;
    ctu3d_body<T, TX, TY, TZ>(a, blockIdx.x, dtd, smem_raw, smax, bad);
    const bool bad_cta = __syncthreads_or(bad) != 0;
    const double m = block_max_t<NT, T>(smax, red);
    finish_step<NT>(m, bad_cta, a, gridDim.x, blockIdx.x, dtd, true, &s_last);
}

}  // namespace hydro
