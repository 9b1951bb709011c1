// step3d.cuh -- one unsplit finite-volume step of the 3D compressible Euler
// equations, fused into a single kernel.
//
// Decomposition (2.5-D blocking): a CTA owns a TX x TY column of cells in the
// x-y plane and marches up a chunk of z planes [z0, z1).  Per plane p it
//   1. stages the next plane of U^n with a depth-2 x-y halo in shared
//      memory, boundary conditions applied by index mapping, converted to
//      primitives (a ring of the planes p-1, p, p+1, and where shared memory
//      allows a spare slot for p+2, so that this staging and step 2 share
//      one barrier interval);
//   2. computes MC slopes and the MUSCL-Hancock half step of plane p for the
//      cells that own a needed face: the tile plus a one-cell cross-shaped
//      ring; x/y face states go to shared memory, the z face states of the
//      thread's own column stay in registers;
//   3. evaluates each x and y face flux of plane p once (HLLC) and the z
//      flux at p - 1/2 (thread's own column);
//   4. completes plane p-1: flux divergence, gravity sources, store of
//      U^{n+1}, positivity check and the cell's CFL signal speed.
// The only HBM traffic is one read of U^n (plus halo re-reads, mostly L2
// hits) and one write of U^{n+1}.  The CTA max signal speed feeds a
// last-CTA FP64 reduction that sets the next dt on the device.
#pragma once

#include <type_traits>

#include "hydro_device.cuh"
#include "per_device.h"

// Staging depth (template argument AS): with AS the next plane is staged by
// asynchronous global->shared copies (cp.async) issued one plane ahead, so
// that its loads are in flight while the current plane is computed without
// holding them in registers; without it each plane is loaded, then
// converted.  The MUSCL-Hancock step offers both (tile variants 4..7 and
// 0..3) to the autotuner; the other kernels take the precision's default:
// asynchronous for FP64 (+1.4 % measured on GB300, one CTA per SM), none for
// FP32 (its further resident CTAs already hide the loads).  The build option
// HYDRO_ASYNC_STAGING=0 turns the asynchronous path off everywhere.
#ifndef HYDRO_ASYNC_STAGING
#define HYDRO_ASYNC_STAGING 1
#endif

// Build options: minimum resident CTAs per SM asked of the FP64 kernels and
// of the FP32 kernels of up to 256 threads (trade registers for occupancy).
// The FP32 32 x 8 tile asks for three (80 registers, measured +5 % on
// GB300 at 512^3 over two); the other FP32 tiles lose with three.
#ifndef HYDRO_FP64_MIN_CTAS
#define HYDRO_FP64_MIN_CTAS 1
#endif
#ifndef HYDRO_FP32_MIN_CTAS
#define HYDRO_FP32_MIN_CTAS 2
#endif
#ifndef HYDRO_FP32_32X8_MIN_CTAS
#define HYDRO_FP32_32X8_MIN_CTAS 3
#endif
#define HYDRO_STEP3D_MIN_CTAS(T, TX, TY)                                                                 \
    (sizeof(T) == 4 ? ((TX) * (TY) > 256 ? 1 : ((TX) == 32 && (TY) == 8 ? HYDRO_FP32_32X8_MIN_CTAS      \
                                                                          : HYDRO_FP32_MIN_CTAS))      \
                    : HYDRO_FP64_MIN_CTAS)

namespace hydro {

template <typename T, bool HSE, int TX, int TY, int RC = RECON_PLM, bool AS = (sizeof(T) == 8)>
struct Step3DSmem {
    static constexpr int NV = 5;
    // halo depth and primitive ring: PLM needs cells i-2..i+2 for the faces
    // of a face neighbour (ring of planes p-1..p+1), PPM i-3..i+3 (p-2..p+2)
    static constexpr int H = RC == RECON_PPM ? 3 : 2;
    static constexpr int HX = TX + 2 * H, HY = TY + 2 * H;
    // Row stride of the staged planes.  A warp of a 16-wide tile spans two
    // rows; for 4-byte values a stride = 16 (mod 32) puts them on disjoint
    // shared-memory banks.  (8-byte values take one wavefront per row.)
    static constexpr int HXS = (TX == 16 && sizeof(T) == 4) ? 48 : HX;
    static constexpr size_t wx = (size_t)NV * TY * (TX + 2);   // [NV][TY][TX+2]
    static constexpr size_t wy = (size_t)NV * (TY + 2) * TX;   // [NV][TY+2][TX]
    static constexpr size_t fx = (size_t)NV * TY * (TX + 1);   // [NV][TY][TX+1]
    static constexpr size_t fy = (size_t)NV * (TY + 1) * TX;   // [NV][TY+1][TX]
    // conserved values of the next two planes as copied from HBM, per
    // variable either HY x HX mapped cells or HY rows of TX / W + 2 16-byte
    // vectors (W cells each), whichever is larger, rounded to a vector
    static constexpr bool async = HYDRO_ASYNC_STAGING != 0 && AS;
    static constexpr int ctas = HYDRO_STEP3D_MIN_CTAS(T, TX, TY);
    // cells per row vector: 16 bytes, except the FP32 tiles held to 80
    // registers (three CTAs per SM) with synchronous staging, whose four
    // loaded vectors of 16 bytes would spill: 8 bytes there
    static constexpr int VW = sizeof(T) == 8 ? 2 : (async || ctas < 3 ? 4 : 2);
    static constexpr size_t rps0 = (size_t)HY * (HX > TX + 2 * VW ? HX : TX + 2 * VW);
    static constexpr size_t rps = (rps0 + VW - 1) / VW * VW;
    static constexpr size_t raw = async ? 2ull * NV * rps + VW : 0;   // [2][NV][rps], + alignment pad
    // planes the half step reads (p-1..p+1, PPM p-2..p+2), and one spare
    // slot where it fits: the next plane is then converted into the spare
    // slot in the same barrier interval as the half step (spare = true)
    static constexpr int NRS = RC == RECON_PPM ? 5 : 3;
    // staged arrays per plane: the primitives, and for FP64 PLM also 1/rho
    // (computed by the conversion anyway; the half step then needs no FP64
    // reciprocal of its own)
    static constexpr int NVS = (sizeof(T) == 8 && RC == RECON_PLM) ? NV + 1 : NV;
    static constexpr size_t plane = (size_t)NVS * HY * HXS;
    // FP64 PLM: the x and y differences of adjacent staged primitives, each
    // formed once per plane and read by both cells beside it (two planes:
    // the one the half step reads and the next, formed in the same barrier
    // interval).  x: rows -1..TY, faces -2..TX (the face between cells f and
    // f + 1); y: faces -2..TY, columns -1..TX.
    static constexpr bool diffs = sizeof(T) == 8 && RC == RECON_PLM;
    static constexpr size_t dxn = (size_t)NV * (TY + 2) * (TX + 3);
    static constexpr size_t dyn = (size_t)NV * (TY + 3) * (TX + 2);
    static constexpr size_t dif = diffs ? 2 * (dxn + dyn) : 0;
    static constexpr size_t rest = 2 * wx + 2 * wy + fx + fy + dif + raw;
    // (fits: one CTA's limit, and the tile's resident CTAs per SM, each with
    // about 1.5 KB of reserved and static shared memory, in the SM's 228 KB).
    // Measured on GB300: +4..+21 % for the synchronous FP32 tiles and +4 %
    // for FP64 PPM; -5 % for the FP32 32 x 16 tile with asynchronous staging
    // and -0.4 % for the FP64 PLM tiles, which keep the plain ring.
    static constexpr size_t spare_bytes = ((NRS + 1) * plane + rest) * sizeof(T);
    static constexpr bool spare = spare_bytes <= 226 * 1024 && ctas * (spare_bytes + 1536) <= 228 * 1024
                               && (!async || (sizeof(T) == 8 && RC == RECON_PPM));
    static constexpr int NR = NRS + (spare ? 1 : 0);
    static constexpr size_t prim = (size_t)NR * plane;          // [NR][NV][HY][HXS]
    static constexpr size_t elems = prim + rest;
    static constexpr size_t bytes = elems * sizeof(T);
    static_assert(bytes <= 226 * 1024, "shared memory of one CTA");
};

// Asynchronous 4- or 8-byte global->shared copy (cp.async, cached in L1 and
// L2) and the completion of all of this thread's copies.
template <typename T>
__device__ __forceinline__ void cp_async_elem(T *smem_dst, const T *gmem_src)
{
    static_assert(sizeof(T) == 4 || sizeof(T) == 8, "4- or 8-byte elements");
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(d), "l"(gmem_src), "n"(sizeof(T))
                 : "memory");
}
// Asynchronous global->shared copy of N = 8 or 16 bytes (both addresses
// aligned to N).
template <int N>
__device__ __forceinline__ void cp_async_vec(void *smem_dst, const void *gmem_src)
{
    static_assert(N == 8 || N == 16, "8- or 16-byte vectors");
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(d), "l"(gmem_src), "n"(N) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// One CTA's share of a step: tile `tile` (row-major over tiles_x) of the x-y
// plane, z planes [z0, z1), time step dtd.
// On return smax/bad hold this thread's max CFL signal speed and whether one
// of its new cells failed the admissibility check.
// ST selects the update (STAGE_*): the MUSCL-Hancock step; the first
// Runge-Kutta stage U1 = U + dt L(U); or the second, (U0 + U + dt L(U)) / 2
// with U = U1 and U0 = U^n.  The stages have no half-step predictor and
// take the gravity source on the momentum from the stage's own density.
// RC selects the face states: MC-limited linear (RECON_PLM), or piecewise
// parabolic (RECON_PPM, Runge-Kutta stages without background only).
// GZ: gravity along z only (g_x = g_y = 0); the x and y gravity terms, all
// zero, are left out (their FP64 additions of zeros are not folded).
template <typename T, bool HSE, int TX, int TY, int ST = STAGE_HANCOCK, int RC = RECON_PLM,
          bool AS = (sizeof(T) == 8), bool GZ = false>
__device__ __forceinline__ void step3d_body(const StepArgs &a, int tile, int z0, int z1, double dtd,
                                            unsigned char *smem_raw, T &smax, bool &bad)
{
    constexpr int ND = 3, NV = 5, NT = TX * TY;
    static_assert(RC == RECON_PLM || (ST != STAGE_HANCOCK && !HSE), "PPM: method-of-lines stages, no background");
    static_assert(NT >= 32 + TX && TY <= 32, "high-side faces: x on warp 0, y on warp 1");
    using S = Step3DSmem<T, HSE, TX, TY, RC, AS>;
    constexpr bool ASYNC = S::async;
    constexpr int HX = S::HX, HY = S::HY, H = S::H, NR = S::NR;
    // planes staged ahead of the plane whose face states are computed: with
    // the spare ring slot H, one more than the stencil reaches, so that
    // staging plane p + H and the half step of plane p share one barrier
    // interval; without it H - 1 and a barrier between the two
    constexpr bool MERGED = S::spare;
    constexpr int LEAD = MERGED ? H : H - 1;
    T *prim = reinterpret_cast<T *>(smem_raw);
    T *wxl = prim + S::prim, *wxh = wxl + S::wx;
    T *wyl = wxh + S::wx, *wyh = wyl + S::wy;
    T *fxs = wyh + S::wy, *fys = fxs + S::fx;
    T *dif = fys + S::fy;
    // (16-byte aligned: the vector copies land there)
    T *rawbuf = reinterpret_cast<T *>((reinterpret_cast<unsigned long long>(dif + S::dif) + 15ull) & ~15ull);

    const int nx = a.n[0], ny = a.n[1], nz = a.n[2];
    const int tid = threadIdx.x, tx = tid % TX, ty = tid / TX;
    const int x0 = (tile % a.tiles_x) * TX;
    const int y0 = (tile / a.tiles_x) * TY;
    const T *__restrict__ U = static_cast<const T *>(a.U);
    const T *__restrict__ U0 = static_cast<const T *>(a.U0);
    T *__restrict__ Un = static_cast<T *>(a.Unew);
    const long long vs = a.vstride;
    // plane offsets as 32 x 32 -> 64-bit products (a plane holds fewer than
    // 2^31 cells); 64 x 64-bit multiplies would occupy the FP64 pipe
    const int plane = static_cast<int>(a.plane);
    const T dt = T(dtd), hdt = T(0.5) * T(dtd);
    const T gam = arg_t<T>(a.gamma, a.gamma_f);
    const T igm1 = arg_t<T>(1.0 / (a.gamma - 1.0), a.igm1_f);
    const PlaneBGT<T> *bgT = static_cast<const PlaneBGT<T> *>(a.bgT);
    const T inv_dx[3] = {arg_t<T>(a.inv_dx[0], a.inv_dx_f[0]),
                          arg_t<T>(a.inv_dx[1], a.inv_dx_f[1]),
                          arg_t<T>(a.inv_dx[2], a.inv_dx_f[2])};
    const T grav[3] = {arg_t<T>(a.grav[0], a.grav_f[0]),
                        arg_t<T>(a.grav[1], a.grav_f[1]),
                        arg_t<T>(a.grav[2], a.grav_f[2])};

    constexpr int HXS = S::HXS;
    constexpr int NVS = S::NVS;
    auto P = [&](int slot, int q, int hy, int hx) -> T & {
        return prim[((slot * NVS + q) * HY + hy) * HXS + hx];   // 32-bit shared-memory indices
    };

    // ---- stage plane pz (may be a ghost plane) into its ring slot, in two
    // halves: fetch() starts the global loads of the haloed plane (boundary
    // conditions applied by index mapping), store() converts them to
    // primitives in shared memory, negating mirrored momenta.  With ASYNC
    // the loads are cp.async copies into a two-plane shared buffer, issued
    // one plane ahead; each thread converts exactly the elements it copied,
    // so its own wait_group suffices.  A tile whose x halo lies inside the
    // grid (VEC, the same for the whole CTA) fetches its rows as 16-byte
    // vectors (row vector layout: hydro_device.cuh, rows_vectorisable) and
    // stores pairs of cells; the others take one load per cell.  Both give
    // the same primitives (the same conversion of the same values).  The
    // x-y mapping of a thread's elements is the same on every plane and is
    // computed once.
    constexpr int NLOAD = (HX * HY + NT - 1) / NT;
    constexpr int HXY = HX * HY;
    constexpr int W = S::VW;                  // cells per vector
    constexpr int NQ = TX / W + 2;            // vectors per row
    constexpr int NVEC = NQ * HY;
    constexpr int NVL = (NVEC + NT - 1) / NT;
    constexpr int NOFF = NLOAD > NVL ? NLOAD : NVL;
    constexpr int RPS = static_cast<int>(S::rps);
    using V16 = typename RowVec<T, W>::V;
    using P2 = typename RowVec<T, 2>::V;
    static_assert(HXS % 2 == 0, "pairs of staged cells are 2-element aligned");
    const bool vec = H == 2 && rows_vectorisable<T, TX, W>(a.U, nx, vs, x0);
    int xyoff[NOFF];          // mapped in-plane offset of each element (or vector)
    unsigned flips = 0;       // bit 2j: x mirror, bit 2j+1: y mirror
    if (vec) {
#pragma unroll
        for (int j = 0; j < NVL; ++j) {
            const int i = tid + j * NT;
            const int k = i % NQ, hy = i / NQ;
            bool fy = false;
            const int gym = i < NVEC ? map_index(y0 + hy - H, ny, a.bc_lo[1], a.bc_hi[1], fy) : 0;
            xyoff[j] = gym * nx + x0 + W * (k - 1);
            flips |= (fy ? 1u : 0u) << (2 * j + 1);
        }
    } else {
#pragma unroll
        for (int j = 0; j < NLOAD; ++j) {
            const int i = tid + j * NT;
            const int hx = i % HX, hy = i / HX;
            bool fx, fy;
            const int gxm = map_index(x0 + hx - H, nx, a.bc_lo[0], a.bc_hi[0], fx);
            const int gym = map_index(y0 + hy - H, ny, a.bc_lo[1], a.bc_hi[1], fy);
            xyoff[j] = gym * nx + gxm;
            flips |= (fx ? 1u : 0u) << (2 * j);
            flips |= (fy ? 1u : 0u) << (2 * j + 1);
        }
    }
    // conserved -> primitive of one cell (o[NV] = 1/rho where staged)
    auto convert = [&](const T (&v)[NV], bool fx, bool fy, bool fz, T rho_bg, T (&o)[NVS]) {
        const T r = v[0];
        const T m0 = fx ? -v[1] : v[1];
        const T m1 = fy ? -v[2] : v[2];
        const T m2 = fz ? -v[3] : v[3];
        const T rho = HSE ? rho_bg + r : r;
        const T rinv = rcp_t(rho);
        const T m[3] = {m0, m1, m2};
        const T u[3] = {mul_rn(m0, rinv), mul_rn(m1, rinv), mul_rn(m2, rinv)};
        o[0] = r;
        o[1] = u[0];
        o[2] = u[1];
        o[3] = u[2];
        o[4] = pressure_of<T, 3>(m, u, v[4], gam - T(1));
        if constexpr (NVS > NV) o[NV] = rinv;
    };
    // the W cells of vector k of row hy, converted, as pairs (the two FP32
    // cells beyond the halo at either end of the row are dropped)
    auto put_vec = [&](int slot, int i, const V16 (&rv)[NV], bool fy, bool fz, T rho_bg) {
        const int k = i % NQ, hy = i / NQ;
#pragma unroll
        for (int e = 0; e < W; e += 2) {
            const int hx = W * (k - 1) + H + e;
            if (W == 2 || (hx >= 0 && hx < HX)) {
                T va[NV], vb[NV], oa[NVS], ob[NVS];
#pragma unroll
                for (int q = 0; q < NV; ++q) { va[q] = vec_lane<T, W>(rv[q], e); vb[q] = vec_lane<T, W>(rv[q], e + 1); }
                convert(va, false, fy, fz, rho_bg, oa);
                convert(vb, false, fy, fz, rho_bg, ob);
#pragma unroll
                for (int q = 0; q < NVS; ++q) {
                    P2 pr;
                    pr.x = oa[q];
                    pr.y = ob[q];
                    *reinterpret_cast<P2 *>(&P(slot, q, hy, hx)) = pr;
                }
            }
        }
    };
    T raw[ASYNC ? 1 : NLOAD][NV];
    auto fetch = [&](int pz) {
        bool fz;
        const int gz = map_index<true>(pz, nz, a.bc_lo[2], a.bc_hi[2], fz);
        // gz is -2 or -1 below a halo side: signed plane offset
        const T *Up = U + (long long)gz * plane;
        T *rb = rawbuf + ((pz + 4) & 1) * (NV * RPS);
        if constexpr (ASYNC) {
            if (vec) {
#pragma unroll
                for (int j = 0; j < NVL; ++j) {
                    const int i = tid + j * NT;
                    if (i < NVEC) {
#pragma unroll
                        for (int q = 0; q < NV; ++q) cp_async_vec<W * sizeof(T)>(rb + q * RPS + i * W, Up + xyoff[j] + q * vs);
                    }
                }
            } else {
#pragma unroll
                for (int j = 0; j < NLOAD; ++j) {
                    const int i = tid + j * NT;
                    if (i < HXY) {
#pragma unroll
                        for (int q = 0; q < NV; ++q) cp_async_elem(rb + q * RPS + i, Up + xyoff[j] + q * vs);
                    }
                }
            }
            cp_async_commit();
        } else {
#pragma unroll
            for (int j = 0; j < NLOAD; ++j) {
                const int i = tid + j * NT;
                if (i < HXY) {
#pragma unroll
                    for (int q = 0; q < NV; ++q) raw[ASYNC ? 0 : j][q] = Up[xyoff[j] + q * vs];
                }
            }
        }
    };
    auto store = [&](int pz) {
        const int slot = (pz + 2 * NR) % NR;
        const T rho_bg = HSE ? bgT[pz + 2].rho_c : T(0);
        bool fz;
        map_index<true>(pz, nz, a.bc_lo[2], a.bc_hi[2], fz);
        const T *rb = rawbuf + ((pz + 4) & 1) * (NV * RPS);
        if constexpr (ASYNC) cp_async_wait_all();
        if (ASYNC && vec) {
#pragma unroll
            for (int j = 0; j < NVL; ++j) {
                const int i = tid + j * NT;
                if (i < NVEC) {
                    V16 rv[NV];
#pragma unroll
                    for (int q = 0; q < NV; ++q) rv[q] = *reinterpret_cast<const V16 *>(rb + q * RPS + i * W);
                    put_vec(slot, i, rv, (flips >> (2 * j + 1)) & 1u, fz, rho_bg);
                }
            }
            return;
        }
#pragma unroll
        for (int j = 0; j < NLOAD; ++j) {
            const int i = tid + j * NT;
            if (i < HXY) {
                const int hx = i % HX, hy = i / HX;
                T v[NV], o[NVS];
#pragma unroll
                for (int q = 0; q < NV; ++q) v[q] = ASYNC ? rb[q * RPS + i] : raw[ASYNC ? 0 : j][q];
                convert(v, (flips >> (2 * j)) & 1u, (flips >> (2 * j + 1)) & 1u, fz, rho_bg, o);
#pragma unroll
                for (int q = 0; q < NVS; ++q) P(slot, q, hy, hx) = o[q];
            }
        }
    };
    // synchronous staging: a vector tile loads and converts its vectors; the
    // others fetch() and store()
    auto stage_sync = [&](int pz) {
        if (!vec) {
            fetch(pz);
            store(pz);
            return;
        }
        bool fz;
        const int gz = map_index<true>(pz, nz, a.bc_lo[2], a.bc_hi[2], fz);
        const T *Up = U + (long long)gz * plane;
        const int slot = (pz + 2 * NR) % NR;
        const T rho_bg = HSE ? bgT[pz + 2].rho_c : T(0);
        // (one vector's loads in flight at a time where a thread has several:
        // their registers would spill)
#pragma unroll
        for (int j = 0; j < NVL; ++j) {
            const int i = tid + j * NT;
            if (i < NVEC) {
                V16 rv[NV];
#pragma unroll
                for (int q = 0; q < NV; ++q) rv[q] = ld_vec<T, W>(Up + xyoff[j] + q * vs);
                put_vec(slot, i, rv, (flips >> (2 * j + 1)) & 1u, fz, rho_bg);
            }
        }
    };

    // ---- x and y differences of plane pz (FP64 PLM; S::diffs): entry f of
    // a row is P(f + 1) - P(f), the same operands and operation as the
    // slope's own differences, so the slopes keep their bits.  Formed once
    // per face instead of once for each of the two cells beside it.
    constexpr bool DIFFS = S::diffs;
    constexpr int DXR = TX + 3, DYR = TX + 2;
    constexpr int NDX = (TY + 2) * DXR, NDY = (TY + 3) * DYR;
    auto DX = [&](int pz, int q, int cy, int f) -> T & {   // cy in [-1, TY], f in [-2, TX]
        return dif[(pz & 1) * (S::dxn + S::dyn) + (q * (TY + 2) + cy + 1) * DXR + f + 2];
    };
    auto DY = [&](int pz, int q, int f, int cx) -> T & {   // f in [-2, TY], cx in [-1, TX]
        return dif[(pz & 1) * (S::dxn + S::dyn) + S::dxn + (q * (TY + 3) + f + 2) * DYR + cx + 1];
    };
    // Each SM sub-partition (warp mod 4) has its own FP64 unit.  The ring
    // cells' half steps run on warps 2 and 3 (ring_start below), so the
    // differences are formed by warps 0, 1, 4, 5, ... (those with warp mod 4
    // < 2): the four units then carry about the same FP64 work between the
    // barriers.
    static_assert(!DIFFS || NT % 128 == 0, "differences on half of the warps");
    constexpr int NDT = NT / 2;
    const int dlane = ((tid >> 7) << 6) + (tid & 63);   // index among the difference threads
    auto form_diffs = [&](int pz) {
        const int sl = (pz + 2 * NR) % NR;
        if (tid & 64) return;
        for (int i = dlane; i < NDX + NDY; i += NDT) {
            if (i < NDX) {
                const int cy = i / DXR - 1, f = i % DXR - 2;
#pragma unroll
                for (int q = 0; q < NV; ++q)
                    DX(pz, q, cy, f) = P(sl, q, cy + H, f + 1 + H) - P(sl, q, cy + H, f + H);
            } else {
                const int j = i - NDX;
                const int f = j / DYR - 2, cx = j % DYR - 1;
#pragma unroll
                for (int q = 0; q < NV; ++q)
                    DY(pz, q, f, cx) = P(sl, q, f + 1 + H, cx + H) - P(sl, q, f + H, cx + H);
            }
        }
    };

    // ---- slopes + half step of the cell at local (cx, cy) of plane p.
    // OWNZ (FP64, the thread's own column): the z difference below plane p
    // is the one above plane p-1, kept in dz from the previous plane (the
    // same operands, so the same bits) -- one FP64 subtraction and one
    // shared-memory load fewer per variable
    auto predict_g = [&](auto OWNZ, int cx, int cy, int p, T (&w)[NV], T (&dw)[ND][NV], T (&wh)[NV],
                         T (&rp)[ND][4], T (&dz)[NV]) {
        constexpr bool ownz = decltype(OWNZ)::value;
        const int s0 = (p + 2 * NR) % NR, sm = (p - 1 + 2 * NR) % NR, sp = (p + 1 + 2 * NR) % NR;
        const int hx = cx + H, hy = cy + H;
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            const T c = P(s0, q, hy, hx);
            w[q] = c;
            if constexpr (DIFFS) {
                dw[0][q] = mc_slope(DX(p, q, cy, cx - 1), DX(p, q, cy, cx));
                dw[1][q] = mc_slope(DY(p, q, cy - 1, cx), DY(p, q, cy, cx));
            } else {
                dw[0][q] = mc_slope(c - P(s0, q, hy, hx - 1), P(s0, q, hy, hx + 1) - c);
                dw[1][q] = mc_slope(c - P(s0, q, hy - 1, hx), P(s0, q, hy + 1, hx) - c);
            }
            if constexpr (ownz) {
                const T dr = P(sp, q, hy, hx) - c;
                dw[2][q] = mc_slope(dz[q], dr);
                dz[q] = dr;
            } else {
                dw[2][q] = mc_slope(c - P(sm, q, hy, hx), P(sp, q, hy, hx) - c);
            }
        }
        const CellBG<T> bg = cell_bg<T, HSE>(bgT, p);
        if constexpr (ST == STAGE_HANCOCK) {
            if constexpr (NVS > NV)
                hancock<T, ND, HSE, GZ, true>(w, dw, wh, rp, hdt, inv_dx, gam, grav, bg, P(s0, NV, hy, hx));
            else
                hancock<T, ND, HSE, GZ>(w, dw, wh, rp, hdt, inv_dx, gam, grav, bg);
        } else {
            mol_faces<T, ND, HSE>(w, dw, bg, rp);
#pragma unroll
            for (int q = 0; q < NV; ++q) wh[q] = w[q];
        }
    };
    constexpr bool OWNZ = sizeof(T) == 8 && RC == RECON_PLM;
    T dz[NV];
    auto predict = [&](int cx, int cy, int p, T (&w)[NV], T (&dw)[ND][NV], T (&wh)[NV], T (&rp)[ND][4]) {
        predict_g(std::false_type{}, cx, cy, p, w, dw, wh, rp, dz);
    };

    // ---- PPM face states of the cell at local (cx, cy) of plane p along
    // axis d for variable q.  The limited faces lie between the cell and its
    // neighbours, so positive densities and pressures stay positive and the
    // positivity fallback of the linear states is never needed.
    auto ppm_dir = [&](int cx, int cy, int p, int d, int q, T &lo, T &hi) {
        const int hx = cx + H, hy = cy + H;
        T v[5];
#pragma unroll
        for (int k = -2; k <= 2; ++k) {
            if (d == 0) v[k + 2] = P((p + 2 * NR) % NR, q, hy, hx + k);
            else if (d == 1) v[k + 2] = P((p + 2 * NR) % NR, q, hy + k, hx);
            else v[k + 2] = P((p + k + 2 * NR) % NR, q, hy, hx);
        }
        const T sm = mc_slope(v[1] - v[0], v[2] - v[1]);
        const T s0 = mc_slope(v[2] - v[1], v[3] - v[2]);
        const T sp = mc_slope(v[3] - v[2], v[4] - v[3]);
        ppm_faces(v[1], v[2], v[3], sm, s0, sp, lo, hi);
    };

    auto WX = [&](T *base, int q, int cy, int cx) -> T & {   // cx in [-1, TX]
        return base[(q * TY + cy) * (TX + 2) + cx + 1];
    };
    auto WY = [&](T *base, int q, int cy, int cx) -> T & {   // cy in [-1, TY]
        return base[(q * (TY + 2) + cy + 1) * TX + cx];
    };
    auto FX = [&](int q, int cy, int fxi) -> T & { return fxs[(q * TY + cy) * (TX + 1) + fxi]; };
    auto FY = [&](int q, int fyi, int cx) -> T & { return fys[(q * (TY + 1) + fyi) * TX + cx]; };

    // register pipeline of the thread's own column
    T ztop_prev[NV], fz_prev[NV], div_prev[NV];
    T msrc_prev = T(0);
#pragma unroll
    for (int q = 0; q < NV; ++q) { ztop_prev[q] = T(0); fz_prev[q] = T(0); div_prev[q] = T(0); }
    smax = T(0);
    bad = false;
    const int gx = x0 + tx, gy = y0 + ty;
    const bool own = gx < nx && gy < ny;
    const int own_off = gy * nx + gx;   // the thread's cell within a plane

    // planes z0-H .. z0+LEAD-2 before the march; iteration p stages p+LEAD
    for (int pz = z0 - H; pz <= z0 + LEAD - 2; ++pz) {
        if constexpr (ASYNC) {
            fetch(pz);
            store(pz);
        } else {
            stage_sync(pz);
        }
    }
    __syncthreads();
    if constexpr (ASYNC) fetch(z0 + LEAD - 1);
    if constexpr (DIFFS) {
        form_diffs(z0 - 1);
        __syncthreads();
    }
    if constexpr (OWNZ) {
        // the own column's z difference below plane z0-1 (planes staged above)
#pragma unroll
        for (int q = 0; q < NV; ++q)
            dz[q] = P((z0 - 1 + 2 * NR) % NR, q, ty + H, tx + H) - P((z0 - 2 + 2 * NR) % NR, q, ty + H, tx + H);
    }
    for (int p = z0 - 1; p <= z1; ++p) {
        // Phase 1: convert plane p+LEAD into its ring slot, then compute the
        // half step of plane p.  MERGED: no barrier between the two (the
        // half step reads the planes p-1..p+1 (PPM p-2..p+2), staged in
        // earlier iterations, not the slot being filled), nor before them
        // (the update of plane p-1 ending the previous iteration touches
        // neither the ring nor the face states).
        // (the last plane any half step reads is z1 + H - 1: the stencil's
        // reach above plane z1)
        if constexpr (ASYNC) {
            // plane p+LEAD was requested one iteration ago; request the next
            // one into the buffer the previous plane used (each thread
            // converts the elements it copied itself)
            if (p + LEAD <= z1 + H - 1) store(p + LEAD);
            if (p + LEAD + 1 <= z1 + H - 1) fetch(p + LEAD + 1);
        } else if (p + LEAD <= z1 + H - 1) {
            stage_sync(p + LEAD);
        }
        if constexpr (!MERGED) __syncthreads();
        const bool xy = (p >= z0 && p < z1);
        // the plane completed at the end of this iteration is p-1: start its
        // own-cell loads now so that they overlap the half step and fluxes
        const bool fin = p > z0 && own;
        T ufin[NV], u0fin[NV];
        T bgB = T(0), bgR = T(0), bgP = T(0);
        if (fin) {
            const long long c = (long long)(p - 1) * plane + own_off;
#pragma unroll
            for (int q = 0; q < NV; ++q) ufin[q] = U[c + q * vs];
            if constexpr (ST == STAGE_RK2) {
#pragma unroll
                for (int q = 0; q < NV; ++q) u0fin[q] = U0[c + q * vs];
            }
            if constexpr (HSE) {
                bgB = bgT[p + 1].B;
                bgR = bgT[p + 1].rho_c;
                bgP = bgT[p + 1].p_c;
            }
        }

        // ---- step 2: half step; own cell first (z faces kept in registers)
        T zlo[NV], ztop[NV];
        if constexpr (RC == RECON_PPM) {
#pragma unroll
            for (int q = 0; q < NV; ++q) ppm_dir(tx, ty, p, 2, q, zlo[q], ztop[q]);
            if (xy) {
#pragma unroll
                for (int q = 0; q < NV; ++q) {
                    T lo, hi;
                    ppm_dir(tx, ty, p, 0, q, lo, hi);
                    WX(wxl, q, ty, tx) = lo;
                    WX(wxh, q, ty, tx) = hi;
                    ppm_dir(tx, ty, p, 1, q, lo, hi);
                    WY(wyl, q, ty, tx) = lo;
                    WY(wyh, q, ty, tx) = hi;
                }
            }
        } else {
            T w[NV], dw[ND][NV], wh[NV], rp[ND][4];
            if constexpr (OWNZ) predict_g(std::true_type{}, tx, ty, p, w, dw, wh, rp, dz);
            else predict(tx, ty, p, w, dw, wh, rp);
#pragma unroll
            for (int q = 0; q < NV; ++q) {
                zlo[q] = face_value<T, ND>(q, 2, false, wh, dw, rp);
                ztop[q] = face_value<T, ND>(q, 2, true, wh, dw, rp);
            }
            if (xy) {
#pragma unroll
                for (int q = 0; q < NV; ++q) {
                    WX(wxl, q, ty, tx) = face_value<T, ND>(q, 0, false, wh, dw, rp);
                    WX(wxh, q, ty, tx) = face_value<T, ND>(q, 0, true, wh, dw, rp);
                    WY(wyl, q, ty, tx) = face_value<T, ND>(q, 1, false, wh, dw, rp);
                    WY(wyh, q, ty, tx) = face_value<T, ND>(q, 1, true, wh, dw, rp);
                }
            }
        }
        if (xy) {
            // ring cells: x = -1 and x = TX (rows 0..TY-1), y = -1 and y = TY
            // (columns 0..TX-1); only their face toward the tile is needed
            constexpr int NRING = 2 * TY + 2 * TX;
            // (FP64: from warp 2 on, see form_diffs)
            const int ring_start = DIFFS ? rotated_start<NT>(tid) : tid;
            for (int i = ring_start; i < NRING; i += NT) {
                int cx, cy;
                bool xside;
                if (i < 2 * TY) { xside = true; cy = i >> 1; cx = (i & 1) ? TX : -1; }
                else { xside = false; const int j = i - 2 * TY; cx = j >> 1; cy = (j & 1) ? TY : -1; }
                if constexpr (RC == RECON_PPM) {
#pragma unroll
                    for (int q = 0; q < NV; ++q) {
                        T lo, hi;
                        ppm_dir(cx, cy, p, xside ? 0 : 1, q, lo, hi);
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
                predict(cx, cy, p, w, dw, wh, rp);
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
        }
        // the next plane's differences (staged and visible since the last
        // barrier) for the next iteration's half step
        if constexpr (DIFFS)
            if (p + 1 <= z1) form_diffs(p + 1);
        __syncthreads();

        // ---- step 3: face fluxes.  Each thread evaluates the low x face and
        // the low y face of its own cell and the z face p - 1/2 of its
        // column as one straight-line block (three independent HLLC solves
        // the scheduler can interleave); the TY + TX high-side faces of the
        // tile follow in a short second pass.  Reflecting walls replace the
        // far-side state by the mirror of the near side's (by selects).
        const T rb_c = HSE ? bgT[p + 2].rho_c : T(0);
        const T pb_c = HSE ? bgT[p + 2].p_c : T(0);
        const T rb_f = HSE ? bgT[p + 2].rho_f : T(0);
        const T pb_f = HSE ? bgT[p + 2].p_f : T(0);
        const bool wall_zlo = p == 0 && a.bc_lo[2] == BC_REFLECT;
        const bool wall_zhi = p == nz && a.bc_hi[2] == BC_REFLECT;
        auto z_states = [&](T (&wl)[NV], T (&wr)[NV]) {
#pragma unroll
            for (int q = 0; q < NV; ++q) {
                const T sgn = q == 3 ? T(-1) : T(1);
                wl[q] = wall_zlo ? sgn * zlo[q] : ztop_prev[q];
                wr[q] = wall_zhi ? sgn * ztop_prev[q] : zlo[q];
            }
        };
        T fz[NV];
        if (xy) {
            T wlx[NV], wrx[NV], wly[NV], wry[NV], wlz[NV], wrz[NV], fxv[NV], fyv[NV];
            // the low face of this cell is a wall when it sits on the domain's
            // low boundary, or on the high boundary (ragged tile: the cell is
            // the first one past the domain)
            // a tile away from every reflecting wall (the common case, the
            // same for the whole CTA) takes the states without the selects
            const bool wall_tile = (a.bc_lo[0] == BC_REFLECT && x0 == 0) || (a.bc_hi[0] == BC_REFLECT && x0 + TX >= nx)
                                || (a.bc_lo[1] == BC_REFLECT && y0 == 0) || (a.bc_hi[1] == BC_REFLECT && y0 + TY >= ny)
                                || wall_zlo || wall_zhi;
            if (!wall_tile) {
#pragma unroll
                for (int q = 0; q < NV; ++q) {
                    wlx[q] = WX(wxh, q, ty, tx - 1);
                    wrx[q] = WX(wxl, q, ty, tx);
                    wly[q] = WY(wyh, q, ty - 1, tx);
                    wry[q] = WY(wyl, q, ty, tx);
                    wlz[q] = ztop_prev[q];
                    wrz[q] = zlo[q];
                }
            } else {
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
                z_states(wlz, wrz);
            }
            hllc<T, ND, 0, HSE>(wlx, wrx, rb_c, pb_c, gam, igm1, fxv);
            hllc<T, ND, 1, HSE>(wly, wry, rb_c, pb_c, gam, igm1, fyv);
            hllc<T, ND, 2, HSE>(wlz, wrz, rb_f, pb_f, gam, igm1, fz);
#pragma unroll
            for (int q = 0; q < NV; ++q) {
                FX(q, ty, tx) = fxv[q];
                FY(q, ty, tx) = fyv[q];
            }
            // high-side faces of the tile: x face TX of each row, y face TY
            // of each column
            // Tiles of up to 256 threads (several CTAs per SM): x faces on
            // warp 0, y faces on warp 1, so that no warp runs both divergent
            // paths (fewer issue slots; +3 % measured).  512-thread tiles keep
            // them packed on the first TX + TY threads, which measured faster
            // there (the other form compiled to fewer registers and less ILP).
            constexpr bool split = NT <= 256;
            if (split ? (tid < TY || (tid >= 32 && tid < 32 + TX)) : tid < TY + TX) {
                const bool isx = tid < TY;
                const int r = isx ? tid : (split ? tid - 32 : tid - TY);
                T wl[NV], wr[NV], f[NV];
                if (isx) {
                    const bool wall = x0 + TX == nx && a.bc_hi[0] == BC_REFLECT;
#pragma unroll
                    for (int q = 0; q < NV; ++q) {
                        wl[q] = WX(wxh, q, r, TX - 1);
                        wr[q] = wall ? (q == 1 ? -wl[q] : wl[q]) : WX(wxl, q, r, TX);
                    }
                    hllc<T, ND, 0, HSE>(wl, wr, rb_c, pb_c, gam, igm1, f);
#pragma unroll
                    for (int q = 0; q < NV; ++q) FX(q, r, TX) = f[q];
                } else {
                    const bool wall = y0 + TY == ny && a.bc_hi[1] == BC_REFLECT;
#pragma unroll
                    for (int q = 0; q < NV; ++q) {
                        wl[q] = WY(wyh, q, TY - 1, r);
                        wr[q] = wall ? (q == 2 ? -wl[q] : wl[q]) : WY(wyl, q, TY, r);
                    }
                    hllc<T, ND, 1, HSE>(wl, wr, rb_c, pb_c, gam, igm1, f);
#pragma unroll
                    for (int q = 0; q < NV; ++q) FY(q, TY, r) = f[q];
                }
            }
        } else if (p == z1) {
            T wlz[NV], wrz[NV];
            z_states(wlz, wrz);
            hllc<T, ND, 2, HSE>(wlz, wrz, rb_f, pb_f, gam, igm1, fz);
        } else {
#pragma unroll
            for (int q = 0; q < NV; ++q) fz[q] = T(0);
        }
        __syncthreads();

        // ---- step 4: complete plane p-1 (an output plane when p > z0)
        if (fin) {
            const int k = p - 1;
            const long long c = (long long)k * plane + own_off;
            T u[NV];
#pragma unroll
            for (int q = 0; q < NV; ++q) u[q] = ufin[q];
            T du[NV];
#pragma unroll
            for (int q = 0; q < NV; ++q) du[q] = -(div_prev[q] + (fz[q] - fz_prev[q]) * inv_dx[2]);
            const T msrc = GZ ? grav[2] * T(0.5) * (fz_prev[0] + fz[0])
                              : msrc_prev + grav[2] * T(0.5) * (fz_prev[0] + fz[0]);
            const T r_old = u[0];
            const T r_new = r_old + dt * du[0];
            u[0] = r_new;
            // gravity on the momentum: time-centred density (MUSCL-Hancock)
            // or the stage's density (Runge-Kutta stages)
            // (the half of the time-centred density is folded into g / 2)
            const T rsum = ST == STAGE_HANCOCK ? r_old + r_new : r_old;
#pragma unroll
            for (int d = 0; d < ND; ++d) {
                if (GZ && d < 2) {
                    u[1 + d] += dt * du[1 + d];
                } else {
                    T src = (ST == STAGE_HANCOCK ? T(0.5) * grav[d] : grav[d]) * rsum;
                    if (HSE && d == 2) src -= bgB;
                    u[1 + d] += dt * (du[1 + d] + src);
                }
            }
            u[4] += dt * (du[4] + msrc);
            if constexpr (ST == STAGE_RK2) {
#pragma unroll
                for (int q = 0; q < NV; ++q) u[q] = T(0.5) * (u0fin[q] + u[q]);
            }
#pragma unroll
            for (int q = 0; q < NV; ++q) Un[c + q * vs] = u[q];
            // CFL signal speed and admissibility of the new state
            const T rho = HSE ? bgR + u[0] : u[0];
            const T rinv = rcp_t(rho);
            const T pp = (gam - T(1)) * (u[4] - half_nonneg(u[1] * u[1] + u[2] * u[2] + u[3] * u[3]) * rinv);
            const T pres = HSE ? bgP + pp : pp;
            const T gp = gam * pres;
            const T cs = gp * rsqrt_t(gp * rho);
            const T s = signal_speed<T, 3>(u + 1, rinv, cs, inv_dx);
            if (!positive(rho) || !positive(pres) || !isfinite(s)) bad = true;
            else smax = max_t(smax, s);
        }
        if (xy) {
            T dv[NV];
#pragma unroll
            for (int q = 0; q < NV; ++q)
                dv[q] = (FX(q, ty, tx + 1) - FX(q, ty, tx)) * inv_dx[0]
                      + (FY(q, ty + 1, tx) - FY(q, ty, tx)) * inv_dx[1];
#pragma unroll
            for (int q = 0; q < NV; ++q) div_prev[q] = dv[q];
            if constexpr (!GZ)
                msrc_prev = grav[0] * T(0.5) * (FX(0, ty, tx) + FX(0, ty, tx + 1))
                          + grav[1] * T(0.5) * (FY(0, ty, tx) + FY(0, ty + 1, tx));
        }
#pragma unroll
        for (int q = 0; q < NV; ++q) { ztop_prev[q] = ztop[q]; fz_prev[q] = fz[q]; }
    }

}

template <typename T, bool HSE, int TX, int TY, int ST = STAGE_HANCOCK, int RC = RECON_PLM,
          bool AS = (sizeof(T) == 8), bool GZ = false>
__global__ void __launch_bounds__(TX * TY, HYDRO_STEP3D_MIN_CTAS(T, TX, TY)) step3d_kernel(const StepArgs a)
{
    constexpr int NT = TX * TY;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[32];
    __shared__ int s_last;
    const int tile = blockIdx.x, chunk = blockIdx.y;
    // time control: dt from the device block, clamped to t_end (both
    // Runge-Kutta stages read the same block: the first stage leaves it
    // unchanged apart from its error bits)
    const double t_now = a.ctrl->t;
    const double dt_cfl = a.ctrl->dt_next;
    // frozen (time at t_end, step limit reached, or error state): nothing
    // moves; the host finds the current buffer from the step count
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
        step3d_body<T, HSE, TX, TY, ST, RC, AS, GZ>(a, t, z0, z1, dtd, smem_raw, sm, bd);
        smax = max_t(smax, sm);
        bad = bad || bd;
    }
    const bool bad_cta = __syncthreads_or(bad) != 0;
    if constexpr (ST == STAGE_RK1) {
        // the intermediate state only raises error bits; dt and time move
        // at the end of the second stage
        if (bad_cta && threadIdx.x == 0) atomicOr(&a.ctrl->err_new, 1);
        return;
    }
    const double m = block_max_t<NT, T>(smax, red);
    finish_step<NT>(m, bad_cta, a, gridDim.x * gridDim.y, blockIdx.x + blockIdx.y * gridDim.x, dtd,
                    true, &s_last);
}

// Persistent batched step: a fixed grid claims the items of all instances
// from the queue's 3D list (largest first).  Each instance keeps its own
// time-control block; the CTA that completes the instance's last item sets
// that instance's next dt (per-instance CFL).  A frozen instance (step limit
// reached, or its error state) is skipped: its state stays where it is.
template <typename T, bool HSE, int TX, int TY, bool AS = (sizeof(T) == 8)>
__global__ void __launch_bounds__(TX * TY, HYDRO_STEP3D_MIN_CTAS(T, TX, TY))
step3d_batch_kernel(const BatchInst *__restrict__ insts, BatchQueue *q, int parity)
{
    constexpr int NT = TX * TY;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[32];
    __shared__ int s_last, s_it;
    __shared__ StepArgs sa;
    const BatchItem *items = q->items[0];
    for (;;) {
        const int it = claim_item(q, 0, parity, &s_it);
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
            const int z0 = w.chunk * sa.zchunk;
            step3d_body<T, HSE, TX, TY, STAGE_HANCOCK, RECON_PLM, AS>(sa, w.tile, z0, min(z0 + sa.zchunk, sa.n[2]),
                                                                      dtd, smem_raw, smax,
                                                                      bad);
            const bool bad_cta = __syncthreads_or(bad) != 0;
            const double m = block_max_t<NT, T>(smax, red);
            finish_step<NT>(m, bad_cta, sa, insts[w.inst].nitems, w.local, dtd, true, &s_last);
        }
        __syncthreads();
    }
}

// Launch of a single-solve step kernel k (TX x TY threads, smem bytes of
// dynamic shared memory).  a.zchunk > 0: the chunked grid `grid` (tiles x
// z-chunks).  a.zchunk <= 0: the balanced grid (PieceIter) -- as many CTAs as
// the device holds resident at once, at most one per plane-tile.  `once`
// and `resident` are the kernel's own per-device set-up records.
template <int TX, int TY, typename K>
cudaError_t launch_step_grid(K k, size_t smem, PerDeviceOnce &once, PerDeviceInt &resident, const StepArgs &a,
                             dim3 grid, cudaStream_t s)
{
    cudaError_t e;
    if (a.zchunk > 0) {
        e = ensure_smem_limit(once, k, smem);
        if (e != cudaSuccess) return e;
        k<<<grid, TX * TY, smem, s>>>(a);
        return cudaGetLastError();
    }
    int g = 0;
    e = persistent_grid(resident, k, smem, TX * TY, &g);
    if (e != cudaSuccess) return e;
    const long long W = (long long)a.tiles_x * ((a.n[1] + TY - 1) / TY) * a.n[2];
    if (g > W) g = static_cast<int>(W);
    k<<<g, TX * TY, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace hydro
