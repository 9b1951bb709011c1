// step2d.cuh -- one unsplit finite-volume step of the 2D compressible Euler
// equations, fused into a single kernel.
//
// A CTA owns a TX x TY tile.  It stages the tile plus a depth-2 halo of U^n
// in shared memory (boundary conditions by index mapping) as primitives,
// computes the MC slopes and MUSCL-Hancock half step of the tile and of the
// one-cell cross-shaped ring whose faces border the tile, evaluates every
// x and y face flux of the tile once (HLLC), then applies the flux
// divergence and gravity sources, stores U^{n+1}, checks admissibility and
// reduces the CFL signal speed (last-CTA FP64 dt on the device).
#pragma once

#include "hydro_device.cuh"
#include "step3d.cuh"   // BatchItem, BatchInst

namespace hydro {

template <typename T, int TX, int TY, int RC = RECON_PLM>
struct Step2DSmem {
    static constexpr int NV = 4;
    static constexpr int H = RC == RECON_PPM ? 3 : 2;   // halo depth
    static constexpr int HX = TX + 2 * H, HY = TY + 2 * H;
    static constexpr size_t prim = (size_t)NV * HY * HX;
    static constexpr size_t wx = (size_t)NV * TY * (TX + 2);
    static constexpr size_t wy = (size_t)NV * (TY + 2) * TX;
    static constexpr size_t fx = (size_t)NV * TY * (TX + 1);
    static constexpr size_t fy = (size_t)NV * (TY + 1) * TX;
    static constexpr size_t elems = prim + 2 * wx + 2 * wy + fx + fy;
    static constexpr size_t bytes = elems * sizeof(T);
};

// One CTA's share of a 2D step: tile `tile` (row-major over tiles_x).  ST
// selects the MUSCL-Hancock step or a Runge-Kutta stage and RC the face
// states (MC-limited linear or PPM) as in step3d_body.
template <typename T, int TX, int TY, int ST = STAGE_HANCOCK, int RC = RECON_PLM>
__device__ __forceinline__ void step2d_body(const StepArgs &a, int tile, double dtd,
                                            unsigned char *smem_raw, T &smax, bool &bad)
{
    constexpr int ND = 2, NV = 4, NT = TX * TY;
    static_assert(RC == RECON_PLM || ST != STAGE_HANCOCK, "PPM: method-of-lines stages");
    using S = Step2DSmem<T, TX, TY, RC>;
    constexpr int HX = S::HX, HY = S::HY, H = S::H;
    T *prim = reinterpret_cast<T *>(smem_raw);
    T *wxl = prim + S::prim, *wxh = wxl + S::wx;
    T *wyl = wxh + S::wx, *wyh = wyl + S::wy;
    T *fxs = wyh + S::wy, *fys = fxs + S::fx;

    const int nx = a.n[0], ny = a.n[1];
    const int tid = threadIdx.x, tx = tid % TX, ty = tid / TX;
    const int x0 = (tile % a.tiles_x) * TX;
    const int y0 = (tile / a.tiles_x) * TY;
    const T *__restrict__ U = static_cast<const T *>(a.U);
    const T *__restrict__ U0 = static_cast<const T *>(a.U0);
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

    auto P = [&](int q, int hy, int hx) -> T & { return prim[(q * HY + hy) * HX + hx]; };
    auto WX = [&](T *base, int q, int cy, int cx) -> T & {
        return base[(q * TY + cy) * (TX + 2) + cx + 1];
    };
    auto WY = [&](T *base, int q, int cy, int cx) -> T & {
        return base[(q * (TY + 2) + cy + 1) * TX + cx];
    };
    auto FX = [&](int q, int cy, int fxi) -> T & { return fxs[(q * TY + cy) * (TX + 1) + fxi]; };
    auto FY = [&](int q, int fyi, int cx) -> T & { return fys[(q * (TY + 1) + fyi) * TX + cx]; };

    // ---- stage the haloed tile as primitives: rows as vectors of W cells
    // where the x halo lies inside the grid (row vector layout:
    // hydro_device.cuh, rows_vectorisable), else one load per cell with
    // boundary index mapping; the same primitives either way
    auto convert = [&](T r, T m0, T m1, T e, int hy, int hx) {
        const T rinv = rcp_t(r);
        const T m[2] = {m0, m1};
        const T u[2] = {mul_rn(m0, rinv), mul_rn(m1, rinv)};
        P(0, hy, hx) = r;
        P(1, hy, hx) = u[0];
        P(2, hy, hx) = u[1];
        P(3, hy, hx) = pressure_of<T, 2>(m, u, e, gam - T(1));
    };
    constexpr int W = 16 / sizeof(T);
    constexpr int NQ = TX / W + 2;
    using V = typename RowVec<T, W>::V;
    if (H == 2 && rows_vectorisable<T, TX, W>(a.U, nx, vs, x0)) {
        for (int i = tid; i < NQ * HY; i += NT) {
            const int k = i % NQ, hy = i / NQ;
            bool fy;
            const int sy = map_index(y0 + hy - H, ny, a.bc_lo[1], a.bc_hi[1], fy);
            const T *src = U + sy * nx + x0 + W * (k - 1);
            V rv[NV];
#pragma unroll
            for (int q = 0; q < NV; ++q) rv[q] = ld_vec<T, W>(src + q * vs);
#pragma unroll
            for (int e = 0; e < W; ++e) {
                const int hx = W * (k - 1) + H + e;
                if (W == 2 || (hx >= 0 && hx < HX)) {
                    const T m1 = vec_lane<T, W>(rv[2], e);
                    convert(vec_lane<T, W>(rv[0], e), vec_lane<T, W>(rv[1], e), fy ? -m1 : m1,
                            vec_lane<T, W>(rv[3], e), hy, hx);
                }
            }
        }
    } else {
        for (int i = tid; i < HX * HY; i += NT) {
            const int hx = i % HX, hy = i / HX;
            bool fx, fy;
            const int sx = map_index(x0 + hx - H, nx, a.bc_lo[0], a.bc_hi[0], fx);
            const int sy = map_index(y0 + hy - H, ny, a.bc_lo[1], a.bc_hi[1], fy);
            const int c = sy * nx + sx;   // a plane holds fewer than 2^31 cells
            const T m0 = U[c + vs], m1 = U[c + 2 * vs];
            convert(U[c], fx ? -m0 : m0, fy ? -m1 : m1, U[c + 3 * vs], hy, hx);
        }
    }
    __syncthreads();

    const CellBG<T> nobg = cell_bg<T, false>(static_cast<const PlaneBGT<T> *>(nullptr), 0);
    auto predict = [&](int cx, int cy, T (&w)[NV], T (&dw)[ND][NV], T (&wh)[NV], T (&rp)[ND][4]) {
        const int hx = cx + H, hy = cy + H;
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            const T c = P(q, hy, hx);
            w[q] = c;
            dw[0][q] = mc_slope(c - P(q, hy, hx - 1), P(q, hy, hx + 1) - c);
            dw[1][q] = mc_slope(c - P(q, hy - 1, hx), P(q, hy + 1, hx) - c);
        }
        if constexpr (ST == STAGE_HANCOCK) {
            hancock<T, ND, false>(w, dw, wh, rp, hdt, inv_dx, gam, grav, nobg);
        } else {
            mol_faces<T, ND, false>(w, dw, nobg, rp);
#pragma unroll
            for (int q = 0; q < NV; ++q) wh[q] = w[q];
        }
    };

    // PPM face states along axis d of variable q (see step3d_body)
    auto ppm_dir = [&](int cx, int cy, int d, int q, T &lo, T &hi) {
        const int hx = cx + H, hy = cy + H;
        T v[5];
#pragma unroll
        for (int k = -2; k <= 2; ++k) v[k + 2] = d == 0 ? P(q, hy, hx + k) : P(q, hy + k, hx);
        const T sm = mc_slope(v[1] - v[0], v[2] - v[1]);
        const T s0 = mc_slope(v[2] - v[1], v[3] - v[2]);
        const T sp = mc_slope(v[3] - v[2], v[4] - v[3]);
        ppm_faces(v[1], v[2], v[3], sm, s0, sp, lo, hi);
    };

    // ---- half step: tile cells, then the cross-shaped ring
    if constexpr (RC == RECON_PPM) {
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            T lo, hi;
            ppm_dir(tx, ty, 0, q, lo, hi);
            WX(wxl, q, ty, tx) = lo;
            WX(wxh, q, ty, tx) = hi;
            ppm_dir(tx, ty, 1, q, lo, hi);
            WY(wyl, q, ty, tx) = lo;
            WY(wyh, q, ty, tx) = hi;
        }
    } else {
        T w[NV], dw[ND][NV], wh[NV], rp[ND][4];
        predict(tx, ty, w, dw, wh, rp);
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            WX(wxl, q, ty, tx) = face_value<T, ND>(q, 0, false, wh, dw, rp);
            WX(wxh, q, ty, tx) = face_value<T, ND>(q, 0, true, wh, dw, rp);
            WY(wyl, q, ty, tx) = face_value<T, ND>(q, 1, false, wh, dw, rp);
            WY(wyh, q, ty, tx) = face_value<T, ND>(q, 1, true, wh, dw, rp);
        }
    }
    constexpr int NRING = 2 * TY + 2 * TX;
    for (int i = tid; i < NRING; i += NT) {
        int cx, cy;
        bool xside;
        if (i < 2 * TY) { xside = true; cy = i >> 1; cx = (i & 1) ? TX : -1; }
        else { xside = false; const int j = i - 2 * TY; cx = j >> 1; cy = (j & 1) ? TY : -1; }
        if constexpr (RC == RECON_PPM) {
#pragma unroll
            for (int q = 0; q < NV; ++q) {
                T lo, hi;
                ppm_dir(cx, cy, xside ? 0 : 1, q, lo, hi);
                if (xside) {
                    if (cx < 0) WX(wxh, q, cy, cx) = hi;
                    else WX(wxl, q, cy, cx) = lo;
                } else {
                    if (cy < 0) WY(wyh, q, cy, cx) = hi;
                    else WY(wyl, q, cy, cx) = lo;
                }
            }
            continue;
        }
        T w[NV], dw[ND][NV], wh[NV], rp[ND][4];
        predict(cx, cy, w, dw, wh, rp);
        if (xside) {
            if (cx < 0) {
#pragma unroll
                for (int q = 0; q < NV; ++q) WX(wxh, q, cy, cx) = face_value<T, ND>(q, 0, true, wh, dw, rp);
            } else {
#pragma unroll
                for (int q = 0; q < NV; ++q) WX(wxl, q, cy, cx) = face_value<T, ND>(q, 0, false, wh, dw, rp);
            }
        } else {
            if (cy < 0) {
#pragma unroll
                for (int q = 0; q < NV; ++q) WY(wyh, q, cy, cx) = face_value<T, ND>(q, 1, true, wh, dw, rp);
            } else {
#pragma unroll
                for (int q = 0; q < NV; ++q) WY(wyl, q, cy, cx) = face_value<T, ND>(q, 1, false, wh, dw, rp);
            }
        }
    }
    __syncthreads();

    // ---- face fluxes: the low x and low y faces of each thread's own cell
    // in one straight-line block, then the high-side faces of the tile.
    // Reflecting walls replace the far-side state by the mirror of the near
    // side's (by selects); a ragged tile's first cell past the domain has
    // the high wall as its low face.
    {
        T wlx[NV], wrx[NV], wly[NV], wry[NV], fxv[NV], fyv[NV];
        const bool xw_lo = x0 + tx == 0 && a.bc_lo[0] == BC_REFLECT;
        const bool xw_hi = x0 + tx == nx && a.bc_hi[0] == BC_REFLECT;
        const bool yw_lo = y0 + ty == 0 && a.bc_lo[1] == BC_REFLECT;
        const bool yw_hi = y0 + ty == ny && a.bc_hi[1] == BC_REFLECT;
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            const T xl = WX(wxh, q, ty, tx - 1), xr = WX(wxl, q, ty, tx);
            wlx[q] = xw_lo ? (q == 1 ? -xr : xr) : xl;
            wrx[q] = xw_hi ? (q == 1 ? -xl : xl) : xr;
            const T yl = WY(wyh, q, ty - 1, tx), yr = WY(wyl, q, ty, tx);
            wly[q] = yw_lo ? (q == 2 ? -yr : yr) : yl;
            wry[q] = yw_hi ? (q == 2 ? -yl : yl) : yr;
        }
        hllc<T, ND, 0, false>(wlx, wrx, T(0), T(0), gam, igm1, fxv);
        hllc<T, ND, 1, false>(wly, wry, T(0), T(0), gam, igm1, fyv);
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            FX(q, ty, tx) = fxv[q];
            FY(q, ty, tx) = fyv[q];
        }
    }
    if (tid < TY + TX) {
        const bool isx = tid < TY;
        const int r = isx ? tid : tid - TY;
        T wl[NV], wr[NV], f[NV];
        if (isx) {
            const bool wall = x0 + TX == nx && a.bc_hi[0] == BC_REFLECT;
#pragma unroll
            for (int q = 0; q < NV; ++q) {
                wl[q] = WX(wxh, q, r, TX - 1);
                wr[q] = wall ? (q == 1 ? -wl[q] : wl[q]) : WX(wxl, q, r, TX);
            }
            hllc<T, ND, 0, false>(wl, wr, T(0), T(0), gam, igm1, f);
#pragma unroll
            for (int q = 0; q < NV; ++q) FX(q, r, TX) = f[q];
        } else {
            const bool wall = y0 + TY == ny && a.bc_hi[1] == BC_REFLECT;
#pragma unroll
            for (int q = 0; q < NV; ++q) {
                wl[q] = WY(wyh, q, TY - 1, r);
                wr[q] = wall ? (q == 2 ? -wl[q] : wl[q]) : WY(wyl, q, TY, r);
            }
            hllc<T, ND, 1, false>(wl, wr, T(0), T(0), gam, igm1, f);
#pragma unroll
            for (int q = 0; q < NV; ++q) FY(q, TY, r) = f[q];
        }
    }
    __syncthreads();

    // ---- update, admissibility, CFL signal speed
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
        const T rsum = ST == STAGE_HANCOCK ? T(0.5) * (r_old + r_new) : r_old;
        u[1] += dt * (du[1] + grav[0] * rsum);
        u[2] += dt * (du[2] + grav[1] * rsum);
        u[3] += dt * (du[3] + msrc);
        if constexpr (ST == STAGE_RK2) {
#pragma unroll
            for (int q = 0; q < NV; ++q) u[q] = T(0.5) * (U0[c + q * vs] + u[q]);
        }
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

template <typename T, int TX, int TY, int ST = STAGE_HANCOCK, int RC = RECON_PLM>
__global__ void __launch_bounds__(TX * TY) step2d_kernel(const StepArgs a)
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
    step2d_body<T, TX, TY, ST, RC>(a, blockIdx.x, dtd, smem_raw, smax, bad);
    const bool bad_cta = __syncthreads_or(bad) != 0;
    if constexpr (ST == STAGE_RK1) {
        if (bad_cta && threadIdx.x == 0) atomicOr(&a.ctrl->err_new, 1);
        return;
    }
    const double m = block_max_t<NT, T>(smax, red);
    finish_step<NT>(m, bad_cta, a, gridDim.x * gridDim.y, blockIdx.x + blockIdx.y * gridDim.x, dtd,
                    true, &s_last);
}

// Persistent batched 2D step over the queue's 2D list of (instance, tile)
// items; the BatchItem/BatchInst layout is shared with the 3D batch (chunk
// unused).  Frozen instances are skipped.
template <typename T, int TX, int TY>
__global__ void __launch_bounds__(TX * TY)
step2d_batch_kernel(const BatchInst *__restrict__ insts, BatchQueue *q, int parity)
{
    constexpr int NT = TX * TY;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[32];
    __shared__ int s_last, s_it;
    __shared__ StepArgs sa;
    const BatchItem *items = q->items[1];
    for (;;) {
        const int it = claim_item(q, 1, parity, &s_it);
        if (it < 0) break;
        const BatchItem w = items[it];
        if (threadIdx.x < (int)(sizeof(StepArgs) / sizeof(int))) {
            reinterpret_cast<int *>(&sa)[threadIdx.x] =
                reinterpret_cast<const int *>(&insts[w.inst].a[parity])[threadIdx.x];
        }
        __syncthreads();
        const double t_now = sa.ctrl->t;
        const double dt_cfl = sa.ctrl->dt_next;
        if (!(t_now >= sa.t_end || sa.ctrl->err != 0 || sa.ctrl->step >= sa.step_end)) {
            const double dtd = (dt_cfl >= sa.t_end - t_now) ? sa.t_end - t_now : dt_cfl;
            T smax;
            bool bad;
            step2d_body<T, TX, TY>(sa, w.tile, dtd, smem_raw, smax, bad);
            const bool bad_cta = __syncthreads_or(bad) != 0;
            const double m = block_max_t<NT, T>(smax, red);
            finish_step<NT>(m, bad_cta, sa, insts[w.inst].nitems, w.local, dtd, true, &s_last);
        }
        __syncthreads();
    }
}

}  // namespace hydro
