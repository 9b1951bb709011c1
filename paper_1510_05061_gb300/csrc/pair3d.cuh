// pair3d.cuh -- the FP32 MUSCL-Hancock step of a 3D grid with two cells per
// thread, in packed f32x2 arithmetic.
//
// Same decomposition as step3d_body (2.5-D blocking: a CTA owns a tile of
// TX x TY cells in the x-y plane and marches up a z-chunk, staging each
// plane with a depth-2 halo as primitives in a shared-memory ring), but each
// thread owns the two x-adjacent cells (2 tx, 2 tx + 1) of its row.  Their
// slopes, half steps, face states, HLLC fluxes (the two low x faces, the
// two low y faces and the two z faces below, as three packed solves) and
// updates are computed together with the pair arithmetic of pair_math.cuh:
// half the FP32 arithmetic instructions, and float2 shared-memory accesses
// where the pair is aligned.  The tile's ring cells and high-side faces are
// evaluated in pairs too (lanes are independent, so every cell and face gets
// the same bits in every tile): x-ring cells and high-side x faces pair the
// two ends of a row or two rows, y-ring cells and high-side y faces are
// aligned pairs.  FP32 only (the FP64 step is bound by its FP64 pipe, which
// has no packed form).
#pragma once

#include "pair_math.cuh"
#include "step3d.cuh"

namespace hydro {

template <bool HSE, int TXP, int TY, int MINB = 1>
struct Pair3DSmem {
    static constexpr int NV = 5, H = 2;
    static constexpr int TX = 2 * TXP;          // cells per tile row
    static constexpr int HX = TX + 2 * H, HY = TY + 2 * H;
    static constexpr int HXS = HX;              // even: the own pair (hx = 2 tx + 2) is 8-byte aligned
    static constexpr int WXS = TX + 4;          // x face states: cell cx in [-1, TX] at cx + 2
    static constexpr int FXS = TX + 2;          // x fluxes: faces 0..TX
    static constexpr size_t wx = (size_t)NV * TY * WXS;        // [NV][TY][WXS]
    static constexpr size_t wy = (size_t)NV * (TY + 2) * TX;   // [NV][TY+2][TX], row cy + 1
    static constexpr size_t fx = (size_t)NV * TY * FXS;        // [NV][TY][FXS]
    static constexpr size_t fy = (size_t)NV * (TY + 1) * TX;   // [NV][TY+1][TX]
    static constexpr size_t plane = (size_t)NV * HY * HXS;
    static constexpr size_t rest = 2 * wx + 2 * wy + fx + fy;
    // a spare ring slot (staging the next plane in the half step's barrier
    // interval) where shared memory allows it for MINB resident CTAs (each
    // with about 1.5 KB of reserved and static shared memory)
    static constexpr bool spare = (4 * plane + rest) * 4 <= 226 * 1024 &&
                                  MINB * ((4 * plane + rest) * 4 + 1536) <= 228 * 1024;
    static constexpr int NR = spare ? 4 : 3;
    // cells per staging row vector (16 bytes)
    static constexpr int VW = 4;
    static constexpr size_t bytes = (NR * plane + rest) * 4;
    static_assert(bytes <= 226 * 1024, "shared memory of one CTA");
};

template <bool HSE, int TXP, int TY, bool GZ, int MINB>
__device__ __forceinline__ void pair3d_body(const StepArgs &a, int tile, int chunk, double dtd,
                                            unsigned char *smem_raw, float &smax, bool &bad)
{
    using S = Pair3DSmem<HSE, TXP, TY, MINB>;
    constexpr int NV = 5, H = 2, NT = TXP * TY;
    constexpr int TX = S::TX, HX = S::HX, HY = S::HY, HXS = S::HXS, NR = S::NR;
    constexpr int WXS = S::WXS, FXS = S::FXS;
    constexpr bool MERGED = S::spare;
    constexpr int LEAD = MERGED ? H : H - 1;
    static_assert(NT >= 64 && TY <= 64 && TXP <= 32, "high-side faces: x pairs on warp 0, y pairs on warp 1");
    float *prim = reinterpret_cast<float *>(smem_raw);
    float *wxl = prim + NR * S::plane, *wxh = wxl + S::wx;
    float *wyl = wxh + S::wx, *wyh = wyl + S::wy;
    float *fxs = wyh + S::wy, *fys = fxs + S::fx;

    const int nx = a.n[0], ny = a.n[1], nz = a.n[2];
    const int tid = threadIdx.x, tx = tid % TXP, ty = tid / TXP;
    const int cx0 = 2 * tx;                      // the pair's first cell in the tile row
    const int x0 = (tile % a.tiles_x) * TX;
    const int y0 = (tile / a.tiles_x) * TY;
    const int z0 = chunk * a.zchunk;
    const int z1 = min(z0 + a.zchunk, nz);
    const float *__restrict__ U = static_cast<const float *>(a.U);
    float *__restrict__ Un = static_cast<float *>(a.Unew);
    const long long vs = a.vstride;
    const int plane = static_cast<int>(a.plane);
    const float dt = float(dtd), hdt = 0.5f * float(dtd);
    const float gam = a.gamma_f, igm1 = a.igm1_f;
    const PlaneBGT<float> *bgT = static_cast<const PlaneBGT<float> *>(a.bgT);
    const float inv_dx[3] = {a.inv_dx_f[0], a.inv_dx_f[1], a.inv_dx_f[2]};
    const float grav[3] = {a.grav_f[0], a.grav_f[1], a.grav_f[2]};

    auto P = [&](int slot, int q, int hy, int hx) -> float & {
        return prim[((slot * NV + q) * HY + hy) * HXS + hx];
    };
    auto P2 = [&](int slot, int q, int hy, int hx) -> f2 & {   // hx even
        return *reinterpret_cast<f2 *>(&prim[((slot * NV + q) * HY + hy) * HXS + hx]);
    };
    auto WX = [&](float *base, int q, int cy, int cx) -> float & { return base[(q * TY + cy) * WXS + cx + 2]; };
    auto WX2 = [&](float *base, int q, int cy, int cx) -> f2 & {   // cx even
        return *reinterpret_cast<f2 *>(&base[(q * TY + cy) * WXS + cx + 2]);
    };
    auto WY = [&](float *base, int q, int cy, int cx) -> float & { return base[(q * (TY + 2) + cy + 1) * TX + cx]; };
    auto WY2 = [&](float *base, int q, int cy, int cx) -> f2 & {
        return *reinterpret_cast<f2 *>(&base[(q * (TY + 2) + cy + 1) * TX + cx]);
    };
    auto FX = [&](int q, int cy, int fi) -> float & { return fxs[(q * TY + cy) * FXS + fi]; };
    auto FX2 = [&](int q, int cy, int fi) -> f2 & { return *reinterpret_cast<f2 *>(&fxs[(q * TY + cy) * FXS + fi]); };
    auto FY2 = [&](int q, int fyi, int cx) -> f2 & {
        return *reinterpret_cast<f2 *>(&fys[(q * (TY + 1) + fyi) * TX + cx]);
    };

    // ---- staging of plane pz (as step3d_body's synchronous staging): row
    // vectors of W cells where the tile's x halo lies inside the grid (VEC,
    // the same for the whole CTA), else one load per cell with boundary
    // index mapping; the same primitives either way
    constexpr int NLOAD = (HX * HY + NT - 1) / NT;
    constexpr int HXY = HX * HY;
    constexpr int W = S::VW;
    constexpr int NQ = TX / W + 2;
    constexpr int NVEC = NQ * HY;
    constexpr int NVL = (NVEC + NT - 1) / NT;
    constexpr int NOFF = NLOAD > NVL ? NLOAD : NVL;
    using VW_t = typename RowVec<float, W>::V;
    const bool vec = rows_vectorisable<float, TX, W>(a.U, nx, vs, x0);
    int xyoff[NOFF];
    unsigned flips = 0;
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
    auto convert = [&](const float (&v)[NV], bool fx, bool fy, bool fz, float rho_bg, float (&o)[NV]) {
        const float r = v[0];
        const float m0 = fx ? -v[1] : v[1];
        const float m1 = fy ? -v[2] : v[2];
        const float m2 = fz ? -v[3] : v[3];
        const float rho = HSE ? rho_bg + r : r;
        const float rinv = rcp_t(rho);
        const float m[3] = {m0, m1, m2};
        const float u[3] = {mul_rn(m0, rinv), mul_rn(m1, rinv), mul_rn(m2, rinv)};
        o[0] = r;
        o[1] = u[0];
        o[2] = u[1];
        o[3] = u[2];
        o[4] = pressure_of<float, 3>(m, u, v[4], gam - 1.0f);
    };
    auto stage = [&](int pz) {
        bool fz;
        const int gz = map_index<true>(pz, nz, a.bc_lo[2], a.bc_hi[2], fz);
        const float *Up = U + (long long)gz * plane;
        const int slot = (pz + 2 * NR) % NR;
        const float rho_bg = HSE ? bgT[pz + 2].rho_c : 0.0f;
        if (vec) {
#pragma unroll
            for (int j = 0; j < NVL; ++j) {
                const int i = tid + j * NT;
                if (i < NVEC) {
                    const int k = i % NQ, hy = i / NQ;
                    const bool fy = (flips >> (2 * j + 1)) & 1u;
                    VW_t rv[NV];
#pragma unroll
                    for (int q = 0; q < NV; ++q) rv[q] = ld_vec<float, W>(Up + xyoff[j] + q * vs);
#pragma unroll
                    for (int e = 0; e < W; e += 2) {
                        const int hx = W * (k - 1) + H + e;   // even
                        if (W == 2 || (hx >= 0 && hx < HX)) {
                            float va[NV], vb[NV], oa[NV], ob[NV];
#pragma unroll
                            for (int q = 0; q < NV; ++q) {
                                va[q] = vec_lane<float, W>(rv[q], e);
                                vb[q] = vec_lane<float, W>(rv[q], e + 1);
                            }
                            convert(va, false, fy, fz, rho_bg, oa);
                            convert(vb, false, fy, fz, rho_bg, ob);
#pragma unroll
                            for (int q = 0; q < NV; ++q) P2(slot, q, hy, hx) = pr(oa[q], ob[q]);
                        }
                    }
                }
            }
            return;
        }
        float raw[NLOAD][NV];
#pragma unroll
        for (int j = 0; j < NLOAD; ++j) {
            const int i = tid + j * NT;
            if (i < HXY) {
#pragma unroll
                for (int q = 0; q < NV; ++q) raw[j][q] = Up[xyoff[j] + q * vs];
            }
        }
#pragma unroll
        for (int j = 0; j < NLOAD; ++j) {
            const int i = tid + j * NT;
            if (i < HXY) {
                const int hx = i % HX, hy = i / HX;
                float o[NV];
                convert(raw[j], (flips >> (2 * j)) & 1u, (flips >> (2 * j + 1)) & 1u, fz, rho_bg, o);
#pragma unroll
                for (int q = 0; q < NV; ++q) P(slot, q, hy, hx) = o[q];
            }
        }
    };

    // ---- slopes + half step of two cells of plane p: the aligned pair at
    // (cx, cy), cx even (float2 loads), or any two cells (a, b) of the plane
    auto finish_predict = [&](int p, f2 (&w)[NV], f2 (&dw)[3][NV], f2 (&wh)[NV]) {
        hancock2<HSE, GZ>(w, dw, wh, hdt, inv_dx, gam, grav, plane_bg<HSE>(bgT, p));
    };
    auto predict_pair = [&](int cx, int cy, int p, f2 (&w)[NV], f2 (&dw)[3][NV], f2 (&wh)[NV]) {
        const int s0 = (p + 2 * NR) % NR, sm = (p - 1 + 2 * NR) % NR, sp = (p + 1 + 2 * NR) % NR;
        const int hx = cx + H, hy = cy + H;
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            const f2 c = P2(s0, q, hy, hx);
            w[q] = c;
            const f2 xl = pr(P(s0, q, hy, hx - 1), c.x), xr = pr(c.y, P(s0, q, hy, hx + 2));
            dw[0][q] = mc_slope2(sub2(c, xl), sub2(xr, c));
            dw[1][q] = mc_slope2(sub2(c, P2(s0, q, hy - 1, hx)), sub2(P2(s0, q, hy + 1, hx), c));
            dw[2][q] = mc_slope2(sub2(c, P2(sm, q, hy, hx)), sub2(P2(sp, q, hy, hx), c));
        }
        finish_predict(p, w, dw, wh);
    };
    auto predict_two = [&](int cxa, int cya, int cxb, int cyb, int p, f2 (&w)[NV], f2 (&dw)[3][NV], f2 (&wh)[NV]) {
        const int s0 = (p + 2 * NR) % NR, sm = (p - 1 + 2 * NR) % NR, sp = (p + 1 + 2 * NR) % NR;
        const int ha = cxa + H, va = cya + H, hb = cxb + H, vb = cyb + H;
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            const f2 c = pr(P(s0, q, va, ha), P(s0, q, vb, hb));
            w[q] = c;
            dw[0][q] = mc_slope2(sub2(c, pr(P(s0, q, va, ha - 1), P(s0, q, vb, hb - 1))),
                                 sub2(pr(P(s0, q, va, ha + 1), P(s0, q, vb, hb + 1)), c));
            dw[1][q] = mc_slope2(sub2(c, pr(P(s0, q, va - 1, ha), P(s0, q, vb - 1, hb))),
                                 sub2(pr(P(s0, q, va + 1, ha), P(s0, q, vb + 1, hb)), c));
            dw[2][q] = mc_slope2(sub2(c, pr(P(sm, q, va, ha), P(sm, q, vb, hb))),
                                 sub2(pr(P(sp, q, va, ha), P(sp, q, vb, hb)), c));
        }
        finish_predict(p, w, dw, wh);
    };
    const f2 mhalf = bc(-0.5f), phalf = bc(0.5f);

    // register pipeline of the thread's own column pair
    f2 ztop_prev[NV], fz_prev[NV], div_prev[NV];
    f2 msrc_prev = bc(0.0f);
#pragma unroll
    for (int q = 0; q < NV; ++q) { ztop_prev[q] = bc(0.0f); fz_prev[q] = bc(0.0f); div_prev[q] = bc(0.0f); }
    smax = 0.0f;
    bad = false;
    const int gx = x0 + cx0, gy = y0 + ty;
    const bool own0 = gx < nx && gy < ny, own1 = gx + 1 < nx && gy < ny;
    const int own_off = gy * nx + gx;
    // the own pair read and written as one 8-byte vector per variable (gx is
    // even; with nx and the variable stride even and both buffers 8-byte
    // aligned, so is every pair's offset)
    const bool own_vec = own0 && own1 && nx % 2 == 0 && vs % 2 == 0 &&
                         ((reinterpret_cast<unsigned long long>(U) | reinterpret_cast<unsigned long long>(Un)) & 7ull) == 0;

    for (int pz = z0 - H; pz <= z0 + LEAD - 2; ++pz) stage(pz);
    __syncthreads();
    for (int p = z0 - 1; p <= z1; ++p) {
        if (p + LEAD <= z1 + H - 1) stage(p + LEAD);
        if constexpr (!MERGED) __syncthreads();
        const bool xy = (p >= z0 && p < z1);
        const bool fin = p > z0 && (own0 || own1);
        const bool wall_zlo = p == 0 && a.bc_lo[2] == BC_REFLECT;
        const bool wall_zhi = p == nz && a.bc_hi[2] == BC_REFLECT;

        // ---- step 2: half step of the own pair; its z faces stay in
        // registers and the z flux below plane p is solved right away (it
        // needs no other thread's states), which ends the low z states'
        // lifetime before the x and y solves
        f2 ztop[NV], fz[NV];
        {
            f2 w[NV], dw[3][NV], wh[NV];
            predict_pair(cx0, ty, p, w, dw, wh);
            if (xy) {
#pragma unroll
                for (int q = 0; q < NV; ++q) {
                    WX2(wxl, q, ty, cx0) = fma2(mhalf, dw[0][q], wh[q]);
                    WX2(wxh, q, ty, cx0) = fma2(phalf, dw[0][q], wh[q]);
                    WY2(wyl, q, ty, cx0) = fma2(mhalf, dw[1][q], wh[q]);
                    WY2(wyh, q, ty, cx0) = fma2(phalf, dw[1][q], wh[q]);
                }
            }
            f2 zlo[NV];
#pragma unroll
            for (int q = 0; q < NV; ++q) {
                zlo[q] = fma2(mhalf, dw[2][q], wh[q]);
                ztop[q] = fma2(phalf, dw[2][q], wh[q]);
            }
            if (p >= z0) {
                f2 wlz[NV], wrz[NV];
#pragma unroll
                for (int q = 0; q < NV; ++q) {
                    const f2 sg = bc(q == 3 ? -1.0f : 1.0f);
                    wlz[q] = wall_zlo ? mul2(sg, zlo[q]) : ztop_prev[q];
                    wrz[q] = wall_zhi ? mul2(sg, ztop_prev[q]) : zlo[q];
                }
                const float rb_f = HSE ? bgT[p + 2].rho_f : 0.0f;
                const float pb_f = HSE ? bgT[p + 2].p_f : 0.0f;
                hllc2<2, HSE>(wlz, wrz, rb_f, pb_f, gam, igm1, fz);
            } else {
#pragma unroll
                for (int q = 0; q < NV; ++q) fz[q] = bc(0.0f);
            }
        }
        if (xy) {
            // ring: TY pairs (x = -1, x = TX) of one row, then TX / 2 aligned
            // pairs of row y = -1 and of row y = TY; only the face toward the
            // tile is kept
            constexpr int NRING = TY + TX;
            for (int i = tid; i < NRING; i += NT) {
                f2 w[NV], dw[3][NV], wh[NV];
                if (i < TY) {
                    predict_two(-1, i, TX, i, p, w, dw, wh);
#pragma unroll
                    for (int q = 0; q < NV; ++q) {
                        WX(wxh, q, i, -1) = fmaf(0.5f, dw[0][q].x, wh[q].x);
                        WX(wxl, q, i, TX) = fmaf(-0.5f, dw[0][q].y, wh[q].y);
                    }
                } else {
                    const int j = i - TY;                 // 0 .. TX-1
                    const int cy = (j & 1) ? TY : -1;
                    const int cx = 2 * (j >> 1);
                    predict_pair(cx, cy, p, w, dw, wh);
                    if (cy < 0) {
#pragma unroll
                        for (int q = 0; q < NV; ++q) WY2(wyh, q, cy, cx) = fma2(phalf, dw[1][q], wh[q]);
                    } else {
#pragma unroll
                        for (int q = 0; q < NV; ++q) WY2(wyl, q, cy, cx) = fma2(mhalf, dw[1][q], wh[q]);
                    }
                }
            }
        }
        __syncthreads();

        // ---- step 3: the pair's two low x faces, then its two low y faces
        // (one packed solve each, in turn), then the tile's high-side faces
        // (x: the rows' faces TX two rows at a time on warp 0; y: aligned
        // pairs of row TY on warp 1)
        const float rb_c = HSE ? bgT[p + 2].rho_c : 0.0f;
        const float pb_c = HSE ? bgT[p + 2].p_c : 0.0f;
        if (xy) {
            const bool wall_tile = (a.bc_lo[0] == BC_REFLECT && x0 == 0) || (a.bc_hi[0] == BC_REFLECT && x0 + TX >= nx)
                                || (a.bc_lo[1] == BC_REFLECT && y0 == 0) || (a.bc_hi[1] == BC_REFLECT && y0 + TY >= ny);
            {
                f2 wl[NV], wr[NV], f[NV];
#pragma unroll
                for (int q = 0; q < NV; ++q) {
                    wl[q] = pr(WX(wxh, q, ty, cx0 - 1), WX(wxh, q, ty, cx0));
                    wr[q] = WX2(wxl, q, ty, cx0);
                }
                if (wall_tile) {
                    // a reflecting wall replaces the far-side state by the
                    // mirror image of the near side's, per lane
                    const bool lo0 = gx == 0 && a.bc_lo[0] == BC_REFLECT, lo1 = gx + 1 == 0 && a.bc_lo[0] == BC_REFLECT;
                    const bool hi0 = gx == nx && a.bc_hi[0] == BC_REFLECT, hi1 = gx + 1 == nx && a.bc_hi[0] == BC_REFLECT;
#pragma unroll
                    for (int q = 0; q < NV; ++q) {
                        const float sx = q == 1 ? -1.0f : 1.0f;
                        const f2 l = wl[q], r = wr[q];
                        wl[q] = pr(lo0 ? sx * r.x : l.x, lo1 ? sx * r.y : l.y);
                        wr[q] = pr(hi0 ? sx * l.x : r.x, hi1 ? sx * l.y : r.y);
                    }
                }
                hllc2<0, HSE>(wl, wr, rb_c, pb_c, gam, igm1, f);
#pragma unroll
                for (int q = 0; q < NV; ++q) FX2(q, ty, cx0) = f[q];
            }
            {
                f2 wl[NV], wr[NV], f[NV];
#pragma unroll
                for (int q = 0; q < NV; ++q) {
                    wl[q] = WY2(wyh, q, ty - 1, cx0);
                    wr[q] = WY2(wyl, q, ty, cx0);
                }
                if (wall_tile) {
                    const bool lo = gy == 0 && a.bc_lo[1] == BC_REFLECT, hi = gy == ny && a.bc_hi[1] == BC_REFLECT;
#pragma unroll
                    for (int q = 0; q < NV; ++q) {
                        const f2 sy = bc(q == 2 ? -1.0f : 1.0f);
                        const f2 l = wl[q], r = wr[q];
                        wl[q] = lo ? mul2(sy, r) : l;
                        wr[q] = hi ? mul2(sy, l) : r;
                    }
                }
                hllc2<1, HSE>(wl, wr, rb_c, pb_c, gam, igm1, f);
#pragma unroll
                for (int q = 0; q < NV; ++q) FY2(q, ty, cx0) = f[q];
            }
            if (tid < TY / 2 || (tid >= 32 && tid < 32 + TXP)) {
                f2 wl[NV], wr[NV], f[NV];
                if (tid < TY / 2) {
                    const int ra = tid, rb = tid + TY / 2;    // two rows' faces TX
                    const bool wall = x0 + TX == nx && a.bc_hi[0] == BC_REFLECT;
#pragma unroll
                    for (int q = 0; q < NV; ++q) {
                        wl[q] = pr(WX(wxh, q, ra, TX - 1), WX(wxh, q, rb, TX - 1));
                        wr[q] = wall ? mul2(bc(q == 1 ? -1.0f : 1.0f), wl[q])
                                     : pr(WX(wxl, q, ra, TX), WX(wxl, q, rb, TX));
                    }
                    hllc2<0, HSE>(wl, wr, rb_c, pb_c, gam, igm1, f);
#pragma unroll
                    for (int q = 0; q < NV; ++q) {
                        FX(q, ra, TX) = f[q].x;
                        FX(q, rb, TX) = f[q].y;
                    }
                } else {
                    const int cx = 2 * (tid - 32);
                    const bool wall = y0 + TY == ny && a.bc_hi[1] == BC_REFLECT;
#pragma unroll
                    for (int q = 0; q < NV; ++q) {
                        wl[q] = WY2(wyh, q, TY - 1, cx);
                        wr[q] = wall ? mul2(bc(q == 2 ? -1.0f : 1.0f), wl[q]) : WY2(wyl, q, TY, cx);
                    }
                    hllc2<1, HSE>(wl, wr, rb_c, pb_c, gam, igm1, f);
#pragma unroll
                    for (int q = 0; q < NV; ++q) FY2(q, TY, cx) = f[q];
                }
            }
        }
        __syncthreads();

        // ---- step 4: complete plane p-1 for the own pair
        if (fin) {
            const long long c = (long long)(p - 1) * plane + own_off;
            f2 u[NV], du[NV];
#pragma unroll
            for (int q = 0; q < NV; ++q)
                u[q] = own_vec ? __ldg(reinterpret_cast<const f2 *>(U + c + q * vs))
                               : pr(own0 ? U[c + q * vs] : 0.0f, own1 ? U[c + 1 + q * vs] : 0.0f);
            const float bgB = HSE ? bgT[p + 1].B : 0.0f;
            const float bgR = HSE ? bgT[p + 1].rho_c : 0.0f;
            const float bgP = HSE ? bgT[p + 1].p_c : 0.0f;
            const f2 idz = bc(inv_dx[2]);
#pragma unroll
            for (int q = 0; q < NV; ++q) du[q] = mul2(bc(-1.0f), fma2(sub2(fz[q], fz_prev[q]), idz, div_prev[q]));
            const f2 zmass = mul2(bc(0.5f * grav[2]), add2(fz_prev[0], fz[0]));
            const f2 msrc = GZ ? zmass : add2(msrc_prev, zmass);
            const f2 h = bc(dt);
            const f2 r_old = u[0];
            const f2 r_new = fma2(h, du[0], r_old);
            u[0] = r_new;
            const f2 rsum = mul2(bc(0.5f), add2(r_old, r_new));
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                if (GZ && d < 2) {
                    u[1 + d] = fma2(h, du[1 + d], u[1 + d]);
                } else {
                    f2 src = mul2(bc(grav[d]), rsum);
                    if (HSE && d == 2) src = sub2(src, bc(bgB));
                    u[1 + d] = fma2(h, add2(du[1 + d], src), u[1 + d]);
                }
            }
            u[4] = fma2(h, add2(du[4], msrc), u[4]);
#pragma unroll
            for (int q = 0; q < NV; ++q) {
                if (own_vec) {
                    *reinterpret_cast<f2 *>(Un + c + q * vs) = u[q];
                } else {
                    if (own0) Un[c + q * vs] = u[q].x;
                    if (own1) Un[c + 1 + q * vs] = u[q].y;
                }
            }
            // CFL signal speed and admissibility of the new states
            const f2 rho = HSE ? add2(bc(bgR), u[0]) : u[0];
            const f2 rinv = rcp2(rho);
            const f2 m2 = fma2(u[3], u[3], fma2(u[2], u[2], mul2(u[1], u[1])));
            const f2 pp = mul2(bc(gam - 1.0f), sub2(u[4], mul2(mul2(bc(0.5f), m2), rinv)));
            const f2 pres = HSE ? add2(bc(bgP), pp) : pp;
            const f2 gp = mul2(bc(gam), pres);
            const f2 cs = mul2(gp, rsqrt2(mul2(gp, rho)));
            const f2 vx = abs2(mul2(u[1], rinv)), vy = abs2(mul2(u[2], rinv)), vz = abs2(mul2(u[3], rinv));
            const f2 s = fma2(add2(vz, cs), bc(inv_dx[2]),
                              fma2(add2(vy, cs), bc(inv_dx[1]), mul2(add2(vx, cs), bc(inv_dx[0]))));
            if (own0) {
                if (!(rho.x > 0.0f) || !(pres.x > 0.0f) || !isfinite(s.x)) bad = true;
                else smax = fmaxf(smax, s.x);
            }
            if (own1) {
                if (!(rho.y > 0.0f) || !(pres.y > 0.0f) || !isfinite(s.y)) bad = true;
                else smax = fmaxf(smax, s.y);
            }
        }
        if (xy) {
            const f2 idx = bc(inv_dx[0]), idy = bc(inv_dx[1]);
#pragma unroll
            for (int q = 0; q < NV; ++q) {
                const f2 flo = FX2(q, ty, cx0);
                const f2 fhi = pr(flo.y, FX(q, ty, cx0 + 2));
                div_prev[q] = fma2(sub2(FY2(q, ty + 1, cx0), FY2(q, ty, cx0)), idy, mul2(sub2(fhi, flo), idx));
            }
            if constexpr (!GZ) {
                const f2 flo = FX2(0, ty, cx0);
                const f2 fhi = pr(flo.y, FX(0, ty, cx0 + 2));
                msrc_prev = fma2(bc(0.5f * grav[1]), add2(FY2(0, ty, cx0), FY2(0, ty + 1, cx0)),
                                 mul2(bc(0.5f * grav[0]), add2(flo, fhi)));
            }
        }
#pragma unroll
        for (int q = 0; q < NV; ++q) { ztop_prev[q] = ztop[q]; fz_prev[q] = fz[q]; }
    }
}

template <bool HSE, int TXP, int TY, bool GZ, int MINB = 1>
__global__ void __launch_bounds__(TXP * TY, MINB) step3d_pair_kernel(const StepArgs a)
{
    constexpr int NT = TXP * TY;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[32];
    __shared__ int s_last;
    const int tile = blockIdx.x, chunk = blockIdx.y;
    const double t_now = a.ctrl->t;
    const double dt_cfl = a.ctrl->dt_next;
    // frozen: nothing moves (the host finds the current buffer from the step count)
    if (t_now >= a.t_end || a.ctrl->err != 0 || a.ctrl->step >= a.step_end) return;
    const double dtd = (dt_cfl >= a.t_end - t_now) ? a.t_end - t_now : dt_cfl;
    float smax;
    bool bad;
    pair3d_body<HSE, TXP, TY, GZ, MINB>(a, tile, chunk, dtd, smem_raw, smax, bad);
    const bool bad_cta = __syncthreads_or(bad) != 0;
    const double m = block_max_t<NT, float>(smax, red);
    finish_step<NT>(m, bad_cta, a, gridDim.x * gridDim.y, blockIdx.x + blockIdx.y * gridDim.x, dtd, true,
                    &s_last);
}

}  // namespace hydro
