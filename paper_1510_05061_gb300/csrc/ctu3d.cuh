// ctu3d.cuh -- one step of the corner transport upwind method (Colella
// 1990) for the 3D compressible Euler equations, fused into one kernel.
//
// A CTA owns a TX x TY column of cells and marches up a chunk of z planes
// [z0, z1).  The face states of plane p need first-pass fluxes of the planes
// p-1, p, p+1, so the march keeps two planes of everything in shared memory.
// At step p it
//   1. stages plane p+1 of U^n (depth-2 x-y halo) as primitives (a ring of
//      the planes p-1, p, p+1);
//   2. computes the one-dimensional MUSCL-Hancock face states of plane p
//      (each axis's own A_d term and half a step of gravity; zero slopes for
//      a cell with a non-positive face density or pressure) on the tile and
//      its one-cell ring;
//   3. evaluates the first-pass HLLC fluxes of plane p (x and y faces of the
//      ring) and of the z faces between planes p-1 and p;
//   4. corrects, in conserved variables and each with -dt/(2 dx_e) times the
//      first-pass flux differences across the other two axes, the z states
//      of plane p and the x and y states of plane p-1 (a cell keeps its
//      uncorrected pair when a corrected density or pressure would not be
//      positive);
//   5. evaluates the final HLLC fluxes of plane p-1's x and y faces and of
//      the z face p-1/2 from the corrected states and completes plane p-1:
//      MUSCL-Hancock update and sources, store, CFL signal speed.
// Reflecting walls mirror the near-side state on both passes.
//
// In the hydrostatic-background mode (HSE) the step is the plain one written
// on the perturbations rho', p' of the stored state: the z predictor advects
// the background and takes g rho'/rho - B_k/rho for gravity, the x and y
// predictors take g; the correction acts on the total state of each face
// (the background's density and pressure at that face added), which is the
// same as correcting the perturbation's density and energy with the total
// density in the momentum and kinetic energy; since the first-pass z fluxes
// carry p', the x and y states' z-momentum correction adds the background's
// pressure difference across the cell; HLLC sees total states and its
// normal momentum flux carries p'; the update takes -B_k on the z momentum.
#pragma once

#include <type_traits>

#include "ctu2d.cuh"   // prim_to_cons_t, cons_to_prim_t, predict_axis

namespace hydro {

template <typename T, int TX, int TY>
struct Ctu3DSmem {
    static constexpr int NV = 5;
    static constexpr int HX = TX + 4, HY = TY + 4;
    static constexpr int EX = TX + 2, EY = TY + 2;               // tile plus ring
    static constexpr size_t prim = 3ull * NV * HY * HX;           // planes p-1, p, p+1
    static constexpr size_t st = (size_t)NV * EY * EX;           // one face-state array
    // the six states of one plane, and the corrected z high state (the
    // uncorrected one still feeds the next plane's first-pass z face)
    static constexpr size_t set = 7 * st;
    static constexpr size_t f1x = (size_t)NV * EY * (TX + 1);    // one plane's x faces
    static constexpr size_t f1y = (size_t)NV * (TY + 1) * EX;
    static constexpr size_t f1z = (size_t)NV * EY * EX;
    static constexpr size_t elems = prim + 2 * (set + f1x + f1y + f1z);
    static constexpr size_t bytes = elems * sizeof(T);
    static_assert(bytes <= 226 * 1024, "shared memory of one CTA");
};

// Conserved variables of a face state: density and energy of the
// perturbation, momentum of the total state (HSE: total density rb + w[0]);
// without background the plain conversion.
template <typename T, bool HSE>
__device__ __forceinline__ void prim_to_cons_bg(const T (&w)[5], T rb, T igm1, T (&u)[5])
{
    const T rho = HSE ? rb + w[0] : w[0];
    T ke = T(0);
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        u[1 + e] = rho * w[1 + e];
        ke += w[1 + e] * w[1 + e];
    }
    u[0] = w[0];
    u[4] = w[4] * igm1 + T(0.5) * rho * ke;
}

template <typename T, bool HSE>
__device__ __forceinline__ void cons_to_prim_bg(const T (&u)[5], T rb, T gam, T (&w)[5])
{
    const T rinv = rcp_t(HSE ? rb + u[0] : u[0]);
    T m2 = T(0);
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        w[1 + e] = u[1 + e] * rinv;
        m2 += u[1 + e] * u[1 + e];
    }
    w[0] = u[0];
    w[4] = (gam - T(1)) * (u[4] - T(0.5) * m2 * rinv);
}

// One-dimensional MUSCL-Hancock predictor along axis d of a cell in the
// hydrostatic-background mode: the perturbation's A_d terms with the total
// density and pressure; along z the background's advection and
// g rho'/rho - B/rho, along x and y plain gravity.
template <typename T>
__device__ __forceinline__ void predict_axis_bg(const T (&w)[5], const T (&dwd)[5], int d, T hdt, T inv_dxd,
                                                T gam, const T (&grav)[3], const CellBG<T> &bg, T (&wd)[5])
{
    const T rho = bg.rho + w[0], pr = bg.p + w[4];
    const T un = w[1 + d];
    const T rinv = rcp_t(rho);
    T r[5];
    r[0] = -(un * dwd[0] + rho * dwd[1 + d]) * inv_dxd;
#pragma unroll
    for (int e = 0; e < 3; ++e) r[1 + e] = -un * dwd[1 + e] * inv_dxd;
    r[1 + d] -= dwd[4] * rinv * inv_dxd;
    r[4] = -(un * dwd[4] + gam * pr * dwd[1 + d]) * inv_dxd;
    if (d == 2) {
        r[0] -= w[3] * bg.drho * inv_dxd;
        r[4] -= w[3] * bg.dp * inv_dxd;
        const T rr = w[0] * rinv;
#pragma unroll
        for (int e = 0; e < 3; ++e) r[1 + e] += grav[e] * rr;
        r[3] -= bg.B * rinv;
    } else {
#pragma unroll
        for (int e = 0; e < 3; ++e) r[1 + e] += grav[e];
    }
#pragma unroll
    for (int q = 0; q < 5; ++q) wd[q] = w[q] + hdt * r[q];
}

template <typename T, bool HSE, int TX, int TY>
__device__ __forceinline__ void ctu3d_body(const StepArgs &a, int tile, int z0, int z1, double dtd,
                                           unsigned char *smem_raw, T &smax, bool &bad)
{
    constexpr int ND = 3, NV = 5, NT = TX * TY;
    using S = Ctu3DSmem<T, TX, TY>;
    constexpr int HX = S::HX, HY = S::HY, EX = S::EX, EY = S::EY;
    T *prim = reinterpret_cast<T *>(smem_raw);
    T *sets = prim + S::prim;                        // [2][7][NV][EY][EX]
    T *f1x = sets + 2 * S::set;                      // [2][NV][EY][TX+1]
    T *f1y = f1x + 2 * S::f1x;                       // [2][NV][TY+1][EX]
    T *f1z = f1y + 2 * S::f1y;                       // [2][NV][EY][EX]

    const int nx = a.n[0], ny = a.n[1], nz = a.n[2];
    const int tid = threadIdx.x, tx = tid % TX, ty = tid / TX;
    const int x0 = (tile % a.tiles_x) * TX;
    const int y0 = (tile / a.tiles_x) * TY;
    const T *__restrict__ U = static_cast<const T *>(a.U);
    T *__restrict__ Un = static_cast<T *>(a.Unew);
    const PlaneBGT<T> *bgT = static_cast<const PlaneBGT<T> *>(a.bgT);
    const long long vs = a.vstride;
    const int plane = static_cast<int>(a.plane);
    const int gx = x0 + tx, gy = y0 + ty;
    const bool own = gx < nx && gy < ny;
    const int own_off = gy * nx + gx;
    const T dt = T(dtd), hdt = T(0.5) * T(dtd);
    const T gam = arg_t<T>(a.gamma, a.gamma_f);
    const T igm1 = arg_t<T>(1.0 / (a.gamma - 1.0), a.igm1_f);
    const T inv_dx[3] = {arg_t<T>(a.inv_dx[0], a.inv_dx_f[0]),
                          arg_t<T>(a.inv_dx[1], a.inv_dx_f[1]),
                          arg_t<T>(a.inv_dx[2], a.inv_dx_f[2])};
    const T grav[3] = {arg_t<T>(a.grav[0], a.grav_f[0]),
                        arg_t<T>(a.grav[1], a.grav_f[1]),
                        arg_t<T>(a.grav[2], a.grav_f[2])};
    const T hdt_dx[3] = {hdt * inv_dx[0], hdt * inv_dx[1], hdt * inv_dx[2]};   // dt / (2 dx_e)

    auto P = [&](int slot, int q, int hy, int hx) -> T & { return prim[((slot * NV + q) * HY + hy) * HX + hx]; };
    // face-state array arr of plane parity b: 0..5 = x lo, x hi, y lo, y hi,
    // z lo, z hi (z lo corrected in place once its first-pass face is done),
    // 6 = corrected z hi
    auto SE = [&](int b, int arr, int q, int cy, int cx) -> T & {
        return sets[(((b * 7 + arr) * NV + q) * EY + cy + 1) * EX + cx + 1];
    };
    // first-pass (later final) x faces fi in [0, TX] left of column fi, rows
    // cy in [-1, TY]; y faces fj in [0, TY], columns cx in [-1, TX]; z faces
    // below plane p (parity of p), cells cx, cy in [-1, T]
    auto FX = [&](int b, int q, int cy, int fi) -> T & { return f1x[((b * NV + q) * EY + cy + 1) * (TX + 1) + fi]; };
    auto FY = [&](int b, int q, int fj, int cx) -> T & { return f1y[((b * NV + q) * (TY + 1) + fj) * EX + cx + 1]; };
    auto FZ = [&](int b, int q, int cy, int cx) -> T & { return f1z[((b * NV + q) * EY + cy + 1) * EX + cx + 1]; };

    // ---- stage plane pz (BC by index mapping) as primitives
    auto stage = [&](int pz) {
        const int slot = (pz + 6) % 3;
        bool fz;
        const int sz = map_index(pz, nz, a.bc_lo[2], a.bc_hi[2], fz);
        const T *Up = U + (long long)sz * plane;
        const T rho_bg = HSE ? bgT[pz + 2].rho_c : T(0);
        for (int i = tid; i < HX * HY; i += NT) {
            const int hx = i % HX, hy = i / HX;
            bool fx, fy;
            const int sx = map_index(x0 + hx - 2, nx, a.bc_lo[0], a.bc_hi[0], fx);
            const int sy = map_index(y0 + hy - 2, ny, a.bc_lo[1], a.bc_hi[1], fy);
            const T *src = Up + sy * nx + sx;
            const T r = src[0];
            T m0 = src[vs], m1 = src[2 * vs], m2 = src[3 * vs];
            const T e = src[4 * vs];
            if (fx) m0 = -m0;
            if (fy) m1 = -m1;
            if (fz) m2 = -m2;
            const T rinv = rcp_t(HSE ? rho_bg + r : r);
            P(slot, 0, hy, hx) = r;
            P(slot, 1, hy, hx) = m0 * rinv;
            P(slot, 2, hy, hx) = m1 * rinv;
            P(slot, 3, hy, hx) = m2 * rinv;
            P(slot, 4, hy, hx) = (gam - T(1)) * (e - T(0.5) * (m0 * m0 + m1 * m1 + m2 * m2) * rinv);
        }
    };

    // ---- one-dimensional face states of plane p on the tile and its ring
    auto predict_plane = [&](int p) {
        const int b = p & 1;
        const int s0 = (p + 6) % 3, sm = (p + 5) % 3, sp = (p + 7) % 3;
        const CellBG<T> bg = cell_bg<T, HSE>(bgT, p);
        for (int i = tid; i < EX * EY; i += NT) {
            const int cx = i % EX - 1, cy = i / EX - 1;
            const int hx = cx + 2, hy = cy + 2;
            T w[NV], dw[ND][NV];
#pragma unroll
            for (int q = 0; q < NV; ++q) {
                const T c = P(s0, q, hy, hx);
                w[q] = c;
                dw[0][q] = mc_slope(c - P(s0, q, hy, hx - 1), P(s0, q, hy, hx + 1) - c);
                dw[1][q] = mc_slope(c - P(s0, q, hy - 1, hx), P(s0, q, hy + 1, hx) - c);
                dw[2][q] = mc_slope(c - P(sm, q, hy, hx), P(sp, q, hy, hx) - c);
            }
            T wd[ND][NV];
            // face densities and pressures {rho_lo, rho_hi, p_lo, p_hi} per
            // axis, formed once for the positivity test and stored as faces
            T rp[ND][4];
            bool ok = true;
#pragma unroll
            for (int d = 0; d < ND; ++d) {
                if constexpr (HSE) predict_axis_bg<T>(w, dw[d], d, hdt, inv_dx[d], gam, grav, bg, wd[d]);
                else predict_axis<T, ND>(w, dw[d], d, hdt, inv_dx[d], gam, grav, wd[d]);
                rp[d][0] = wd[d][0] - T(0.5) * dw[d][0];
                rp[d][1] = wd[d][0] + T(0.5) * dw[d][0];
                rp[d][2] = wd[d][NV - 1] - T(0.5) * dw[d][NV - 1];
                rp[d][3] = wd[d][NV - 1] + T(0.5) * dw[d][NV - 1];
                if constexpr (HSE) {
                    // total face density and pressure: the plane's centre
                    // background for x and y, the z faces' own along z
                    const T rlo = d == 2 ? bg.rho_lo : bg.rho, rhi = d == 2 ? bg.rho_hi : bg.rho;
                    const T plo = d == 2 ? bg.p_lo : bg.p, phi = d == 2 ? bg.p_hi : bg.p;
                    ok = ok && positive(rlo + rp[d][0]) && positive(rhi + rp[d][1])
                            && positive(plo + rp[d][2]) && positive(phi + rp[d][3]);
                } else {
                    ok = ok && positive(rp[d][0]) && positive(rp[d][1]) && positive(rp[d][2]) && positive(rp[d][3]);
                }
            }
            if (!ok) {
                // zero slopes: every face takes the cell state plus half a
                // step of gravity (HSE: the z states the MUSCL-Hancock
                // source g rho'/rho - B/rho, the x and y states g)
                T gz[ND];
#pragma unroll
                for (int e = 0; e < ND; ++e) gz[e] = grav[e];
                if constexpr (HSE) {
                    const T rinv = rcp_t(bg.rho + w[0]);
#pragma unroll
                    for (int e = 0; e < ND; ++e) gz[e] = grav[e] * (w[0] * rinv);
                    gz[2] -= bg.B * rinv;
                }
#pragma unroll
                for (int d = 0; d < ND; ++d)
#pragma unroll
                    for (int q = 0; q < NV; ++q) {
                        dw[d][q] = T(0);
                        const T gq = q >= 1 && q <= ND ? (d == 2 ? gz[q - 1] : grav[q - 1]) : T(0);
                        wd[d][q] = w[q] + (q >= 1 && q <= ND ? hdt * gq : T(0));
                    }
#pragma unroll
                for (int d = 0; d < ND; ++d) {
                    rp[d][0] = rp[d][1] = w[0];
                    rp[d][2] = rp[d][3] = w[NV - 1];
                }
            }
#pragma unroll
            for (int d = 0; d < ND; ++d)
#pragma unroll
                for (int q = 0; q < NV; ++q) {
                    const bool rq = q == 0 || q == NV - 1;
                    const int k = q == 0 ? 0 : 2;
                    SE(b, 2 * d, q, cy, cx) = rq ? rp[d][k] : wd[d][q] - T(0.5) * dw[d][q];
                    SE(b, 2 * d + 1, q, cy, cx) = rq ? rp[d][k + 1] : wd[d][q] + T(0.5) * dw[d][q];
                }
        }
    };

    // HLLC from a left and a right state array along axis D; a wall at the
    // face mirrors the near side
    auto hllc_mirror = [&](auto DC, bool w_lo, bool w_hi, const T (&vl)[NV], const T (&vr)[NV], T rb, T pb,
                           T (&f)[NV]) {
        constexpr int D = decltype(DC)::value;
        T wl[NV], wr[NV];
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            wl[q] = w_lo ? (q == 1 + D ? -vr[q] : vr[q]) : vl[q];
            wr[q] = w_hi ? (q == 1 + D ? -vl[q] : vl[q]) : vr[q];
        }
        hllc<T, ND, D, HSE>(wl, wr, rb, pb, gam, igm1, f);
    };
    using D0 = std::integral_constant<int, 0>;
    using D1 = std::integral_constant<int, 1>;
    using D2 = std::integral_constant<int, 2>;
    // x and y faces of plane pl (parity b): the plane's centre background
    auto x_face = [&](int b, int pl, int cy, int fi, T (&f)[NV]) {
        const int gf = x0 + fi;
        T vl[NV], vr[NV];
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            vl[q] = SE(b, 1, q, cy, fi - 1);
            vr[q] = SE(b, 0, q, cy, fi);
        }
        hllc_mirror(D0{}, gf == 0 && a.bc_lo[0] == BC_REFLECT, gf == nx && a.bc_hi[0] == BC_REFLECT, vl, vr,
                    HSE ? bgT[pl + 2].rho_c : T(0), HSE ? bgT[pl + 2].p_c : T(0), f);
    };
    auto y_face = [&](int b, int pl, int fj, int cx, T (&f)[NV]) {
        const int gf = y0 + fj;
        T vl[NV], vr[NV];
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            vl[q] = SE(b, 3, q, fj - 1, cx);
            vr[q] = SE(b, 2, q, fj, cx);
        }
        hllc_mirror(D1{}, gf == 0 && a.bc_lo[1] == BC_REFLECT, gf == ny && a.bc_hi[1] == BC_REFLECT, vl, vr,
                    HSE ? bgT[pl + 2].rho_c : T(0), HSE ? bgT[pl + 2].p_c : T(0), f);
    };
    // z face below plane p between the high state of plane p-1 (array hi: 5
    // first pass, 6 corrected) and the low state of plane p; the face's own
    // background
    auto z_face = [&](int p, int hi, int cy, int cx, T (&f)[NV]) {
        T vl[NV], vr[NV];
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            vl[q] = SE((p - 1) & 1, hi, q, cy, cx);
            vr[q] = SE(p & 1, 4, q, cy, cx);
        }
        hllc_mirror(D2{}, p == 0 && a.bc_lo[2] == BC_REFLECT, p == nz && a.bc_hi[2] == BC_REFLECT, vl, vr,
                    HSE ? bgT[p + 2].rho_f : T(0), HSE ? bgT[p + 2].p_f : T(0), f);
    };

    // transverse correction of both face states of a cell (arrays lo, lo + 1)
    // into arrays dlo, dhi (the uncorrected pair when a corrected density or
    // pressure would not be positive).  rb, pb: the background at the two
    // faces; dmz: the extra z-momentum correction of HSE x and y states.
    auto correct = [&](int b, int lo, int dlo, int dhi, int cy, int cx, const T (&d1)[NV], T k1,
                       const T (&d2)[NV], T k2, const T (&rb)[2], const T (&pb)[2], T dmz) {
        T wc[2][NV];
        bool ok = true;
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            T w[NV], u[NV];
#pragma unroll
            for (int q = 0; q < NV; ++q) w[q] = SE(b, lo + s, q, cy, cx);
            prim_to_cons_bg<T, HSE>(w, rb[s], igm1, u);
#pragma unroll
            for (int q = 0; q < NV; ++q) u[q] -= k1 * d1[q];
#pragma unroll
            for (int q = 0; q < NV; ++q) u[q] -= k2 * d2[q];
            if constexpr (HSE) u[3] -= dmz;
            cons_to_prim_bg<T, HSE>(u, rb[s], gam, wc[s]);
            ok = ok && positive(HSE ? rb[s] + wc[s][0] : wc[s][0])
                    && positive(HSE ? pb[s] + wc[s][NV - 1] : wc[s][NV - 1]);
        }
        if (ok) {
#pragma unroll
            for (int s = 0; s < 2; ++s)
#pragma unroll
                for (int q = 0; q < NV; ++q) SE(b, s ? dhi : dlo, q, cy, cx) = wc[s][q];
        } else if (dhi != lo + 1) {
#pragma unroll
            for (int q = 0; q < NV; ++q) SE(b, dhi, q, cy, cx) = SE(b, lo + 1, q, cy, cx);
        }
    };

    smax = T(0);
    bad = false;
    T fz_prev[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) fz_prev[q] = T(0);

    stage(z0 - 2);
    stage(z0 - 1);
    for (int p = z0 - 1; p <= z1; ++p) {
        const int b = p & 1, bm = (p - 1) & 1;
        // 1.-2. next plane, then the one-dimensional states of plane p
        stage(p + 1);
        __syncthreads();
        predict_plane(p);
        __syncthreads();

        // 3. first-pass fluxes of plane p, and of the z faces below it
        for (int i = tid; i < (TX + 1) * EY; i += NT) {
            const int fi = i % (TX + 1), cy = i / (TX + 1) - 1;
            T f[NV];
            x_face(b, p, cy, fi, f);
#pragma unroll
            for (int q = 0; q < NV; ++q) FX(b, q, cy, fi) = f[q];
        }
        for (int i = rotated_start<NT>(tid); i < EX * (TY + 1); i += NT) {   // second pass off warp 0
            const int cx = i % EX - 1, fj = i / EX;
            T f[NV];
            y_face(b, p, fj, cx, f);
#pragma unroll
            for (int q = 0; q < NV; ++q) FY(b, q, fj, cx) = f[q];
        }
        if (p >= z0) {
            for (int i = tid; i < EX * EY; i += NT) {
                const int cx = i % EX - 1, cy = i / EX - 1;
                T f[NV];
                z_face(p, 5, cy, cx, f);
#pragma unroll
                for (int q = 0; q < NV; ++q) FZ(b, q, cy, cx) = f[q];
            }
        }
        __syncthreads();

        // 4. corrections: z states of plane p (tile cells), x and y states of
        // plane p-1 (its z faces' first-pass fluxes are now both known)
        T rbz[2] = {T(0), T(0)}, pbz[2] = {T(0), T(0)}, rbc[2] = {T(0), T(0)}, pbc[2] = {T(0), T(0)};
        T dmz = T(0);
        if constexpr (HSE) {
            rbz[0] = bgT[p + 2].rho_f; rbz[1] = bgT[p + 3].rho_f;
            pbz[0] = bgT[p + 2].p_f;   pbz[1] = bgT[p + 3].p_f;
            rbc[0] = rbc[1] = bgT[p + 1].rho_c;
            pbc[0] = pbc[1] = bgT[p + 1].p_c;
            dmz = hdt_dx[2] * bgT[p + 1].dp;
        }
        for (int i = tid; i < TX * TY; i += NT) {
            const int cx = i % TX, cy = i / TX;
            T dx1[NV], dy1[NV];
#pragma unroll
            for (int q = 0; q < NV; ++q) {
                dx1[q] = FX(b, q, cy, cx + 1) - FX(b, q, cy, cx);
                dy1[q] = FY(b, q, cy + 1, cx) - FY(b, q, cy, cx);
            }
            correct(b, 4, 4, 6, cy, cx, dx1, hdt_dx[0], dy1, hdt_dx[1], rbz, pbz, T(0));
        }
        const bool out_plane = p - 1 >= z0 && p - 1 < z1;   // plane p-1 is completed now
        if (out_plane) {
            for (int i = tid; i < EX * TY; i += NT) {        // x states: columns -1..TX, tile rows
                const int cx = i % EX - 1, cy = i / EX;
                T dy1[NV], dz1[NV];
#pragma unroll
                for (int q = 0; q < NV; ++q) {
                    dy1[q] = FY(bm, q, cy + 1, cx) - FY(bm, q, cy, cx);
                    dz1[q] = FZ(b, q, cy, cx) - FZ(bm, q, cy, cx);
                }
                correct(bm, 0, 0, 1, cy, cx, dy1, hdt_dx[1], dz1, hdt_dx[2], rbc, pbc, dmz);
            }
            // y states: tile columns, rows -1..TY (second pass off warp 0)
            for (int i = rotated_start<NT>(tid); i < TX * EY; i += NT) {
                const int cx = i % TX, cy = i / TX - 1;
                T dx1[NV], dz1[NV];
#pragma unroll
                for (int q = 0; q < NV; ++q) {
                    dx1[q] = FX(bm, q, cy, cx + 1) - FX(bm, q, cy, cx);
                    dz1[q] = FZ(b, q, cy, cx) - FZ(bm, q, cy, cx);
                }
                correct(bm, 2, 2, 3, cy, cx, dx1, hdt_dx[0], dz1, hdt_dx[2], rbc, pbc, dmz);
            }
        }
        __syncthreads();

        // 5. final fluxes: x and y faces of plane p-1 (over its first-pass
        // arrays), the z face p-1/2 of the own column
        if (out_plane) {
            for (int i = tid; i < (TX + 1) * TY; i += NT) {
                const int fi = i % (TX + 1), cy = i / (TX + 1);
                T f[NV];
                x_face(bm, p - 1, cy, fi, f);
#pragma unroll
                for (int q = 0; q < NV; ++q) FX(bm, q, cy, fi) = f[q];
            }
            for (int i = rotated_start<NT>(tid); i < TX * (TY + 1); i += NT) {
                const int cx = i % TX, fj = i / TX;
                T f[NV];
                y_face(bm, p - 1, fj, cx, f);
#pragma unroll
                for (int q = 0; q < NV; ++q) FY(bm, q, fj, cx) = f[q];
            }
        }
        T fz[NV];
        if (p >= z0) z_face(p, 6, ty, tx, fz);
        __syncthreads();

        // update of plane p-1 (MUSCL-Hancock sources; HSE: -B on the z momentum)
        if (out_plane && own) {
            const long long c = (long long)(p - 1) * plane + own_off;
            T u[NV], du[NV];
#pragma unroll
            for (int q = 0; q < NV; ++q) {
                u[q] = U[c + q * vs];
                du[q] = -((FX(bm, q, ty, tx + 1) - FX(bm, q, ty, tx)) * inv_dx[0]
                          + (FY(bm, q, ty + 1, tx) - FY(bm, q, ty, tx)) * inv_dx[1]
                          + (fz[q] - fz_prev[q]) * inv_dx[2]);
            }
            const T msrc = grav[0] * T(0.5) * (FX(bm, 0, ty, tx) + FX(bm, 0, ty, tx + 1))
                         + grav[1] * T(0.5) * (FY(bm, 0, ty, tx) + FY(bm, 0, ty + 1, tx))
                         + grav[2] * T(0.5) * (fz_prev[0] + fz[0]);
            const T r_old = u[0];
            const T r_new = r_old + dt * du[0];
            u[0] = r_new;
            const T rsum = r_old + r_new;   // (the half is folded into g / 2)
#pragma unroll
            for (int d = 0; d < ND; ++d) {
                T src = (T(0.5) * grav[d]) * rsum;
                if (HSE && d == 2) src -= bgT[p + 1].B;
                u[1 + d] += dt * (du[1 + d] + src);
            }
            u[4] += dt * (du[4] + msrc);
#pragma unroll
            for (int q = 0; q < NV; ++q) Un[c + q * vs] = u[q];
            const T rho = HSE ? bgT[p + 1].rho_c + u[0] : u[0];
            const T rinv = rcp_t(rho);
            const T pp = (gam - T(1)) * (u[4] - half_nonneg(u[1] * u[1] + u[2] * u[2] + u[3] * u[3]) * rinv);
            const T pres = HSE ? bgT[p + 1].p_c + pp : pp;
            const T gp = gam * pres;
            const T cs = gp * rsqrt_t(gp * rho);
            const T s = signal_speed<T, 3>(u + 1, rinv, cs, inv_dx);
            if (!positive(rho) || !positive(pres) || !isfinite(s)) bad = true;
            else smax = max_t(smax, s);
        }
        if (p >= z0) {
#pragma unroll
            for (int q = 0; q < NV; ++q) fz_prev[q] = fz[q];
        }
    }
}

template <typename T, bool HSE, int TX, int TY>
__global__ void __launch_bounds__(TX * TY) ctu3d_kernel(const StepArgs a)
{
    constexpr int NT = TX * TY;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[32];
    __shared__ int s_last;
    const int tile = blockIdx.x, chunk = blockIdx.y;
    const double t_now = a.ctrl->t;
    const double dt_cfl = a.ctrl->dt_next;
    // frozen: nothing moves (the host finds the current buffer from the step count)
    if (t_now >= a.t_end || a.ctrl->err != 0 || a.ctrl->step >= a.step_end) return;
    const double dtd = (dt_cfl >= a.t_end - t_now) ? a.t_end - t_now : dt_cfl;
    T smax = T(0);
    bool bad = false;
    // the CTA's column pieces: one z-chunk of one tile (chunked grid), or
    // its share of the balanced grid (PieceIter)
    PieceIter pieces(a.zchunk, (long long)a.tiles_x * ((a.n[1] + TY - 1) / TY), a.n[2], tile, chunk,
                     gridDim.x, blockIdx.x);
    int t, z0, z1;
    bool first = true;
    while (pieces.next(t, z0, z1)) {
        if (!first) __syncthreads();   // the next piece reuses the shared-memory ring
        first = false;
        T sm;
        bool bd;
        ctu3d_body<T, HSE, TX, TY>(a, t, z0, z1, dtd, smem_raw, sm, bd);
        smax = max_t(smax, sm);
        bad = bad || bd;
    }
    const bool bad_cta = __syncthreads_or(bad) != 0;
    const double m = block_max_t<NT, T>(smax, red);
    finish_step<NT>(m, bad_cta, a, gridDim.x * gridDim.y, blockIdx.x + blockIdx.y * gridDim.x, dtd, true,
                    &s_last);
}

}  // namespace hydro
