// pieces.h -- the column pieces one CTA of a 3D step marches (host and
// device code).
#pragma once

#include <cuda_runtime.h>

namespace hydro {

// The column pieces (tile, [z0, z1)) one CTA of a 3D step marches, in
// marching order, for a grid of T tiles and nz planes:
//  zchunk > 0: the chunked grid, blockIdx = (tile, chunk): one piece.
//  zchunk <= 0: the balanced grid of G CTAs over chunks of Z
//   planes (whole columns, Z = nz, for zchunk 0 or -1, else Z =
//   min(-zchunk, nz)).  The chunks are
//   ordered row by row (row c: planes [cZ, cZ + Z) of every tile) and taken
//   in whole waves while at least G remain -- CTA b takes chunks b, b + G,
//   b + 2G, ... -- so that the resident CTAs march neighbouring tiles at the
//   same heights and find each other's halo rows in L2.  The planes of the
//   remaining (fewer than G) chunks are then split evenly over the G CTAs,
//   each marching its share from its last piece back (the piece that starts
//   lowest first).  When Z divides nz (always for whole columns) every CTA
//   gets the same number of planes (+-1): the launch has no partial last
//   wave.  Otherwise the last row's chunks are shorter, and a CTA taking one
//   of them in a whole wave marches that many planes fewer.
// Every thread of a CTA walks the same pieces.  Host code may walk them
// too (the library's test hook hydro_debug_pieces).
class PieceIter {
public:
    // G: CTAs of the balanced grid, b: this CTA (unused for the chunked grid)
    __host__ __device__ PieceIter(int zchunk, long long tiles, int nz, int tile, int chunk, long long G, long long b)
        : T_(tiles), nz_(nz)
    {
        if (zchunk > 0) {
            mode_ = 0;
            t_ = tile;
            z0_ = chunk * zchunk;
            z1_ = z0_ + zchunk < nz ? z0_ + zchunk : nz;
            return;
        }
        mode_ = 1;
        Z_ = zchunk >= -1 ? nz : (-zchunk < nz ? -zchunk : nz);
        const int nch = (nz + Z_ - 1) / Z_;
        hl_ = nz - (nch - 1) * Z_;
        G_ = G;
        b_ = b;
        const long long I = T_ * nch;
        w_ = I / G_;
        j_ = 0;
        r0_ = w_ * G_;
        const long long last_row = (long long)(nch - 1) * T_;
        nf_ = (last_row < I ? last_row : I) - r0_;
        if (nf_ < 0) nf_ = 0;
        const long long P = nf_ * Z_ + (I - r0_ - nf_) * hl_;
        k0_ = P * b_ / G_;
        k1_ = P * (b_ + 1) / G_;
    }
    // The next piece, or false when the CTA's share is done.
    __host__ __device__ bool next(int &t, int &z0, int &z1)
    {
        if (mode_ == 0) {
            mode_ = 3;
            t = t_;
            z0 = z0_;
            z1 = z1_;
            return true;
        }
        if (mode_ == 1) {
            if (j_ < w_) {
                const long long i = b_ + j_ * G_;
                ++j_;
                const int c = static_cast<int>(i / T_);
                t = static_cast<int>(i % T_);
                z0 = c * Z_;
                z1 = z0 + Z_ < nz_ ? z0 + Z_ : nz_;
                return true;
            }
            mode_ = 2;
        }
        if (mode_ == 2 && k1_ > k0_) {
            // the piece holding share index k1 - 1: chunk i, whose first plane
            // has share index base
            const long long k = k1_ - 1;
            long long i, base;
            if (k < nf_ * Z_) {
                i = r0_ + k / Z_;
                base = (k / Z_) * Z_;
            } else {
                const long long kk = k - nf_ * Z_;
                i = r0_ + nf_ + kk / hl_;
                base = nf_ * Z_ + (kk / hl_) * hl_;
            }
            const long long s = k0_ > base ? k0_ : base;
            const int c = static_cast<int>(i / T_);
            t = static_cast<int>(i % T_);
            z0 = c * Z_ + static_cast<int>(s - base);
            z1 = c * Z_ + static_cast<int>(k1_ - base);
            k1_ = s;
            return true;
        }
        mode_ = 3;
        return false;
    }

private:
    long long T_;
    int nz_, mode_ = 3, t_ = 0, z0_ = 0, z1_ = 0, Z_ = 1, hl_ = 1;
    long long G_ = 1, b_ = 0, w_ = 0, j_ = 0, r0_ = 0, nf_ = 0, k0_ = 0, k1_ = 0;
};

}  // namespace hydro
