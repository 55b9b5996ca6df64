// Register-tiled complex block products shared by the triangular sweeps (ops.cu) and the
// far-field product (far.cu).
//
// A CTA owns an output block of `no` rows x `nrhs` right-hand-side columns.  Each thread
// keeps NT tiles of TR rows x TC columns in registers, placed by tile_rc.  A product step
// takes a staged coefficient block M(row, qq) = Ws[qq * ldw + row] and a staged vector block
// Y(qq, r) = Ys[qq * ysq + r * ysr] and updates acc(row, r) -/+= sum_qq M(row, qq) Y(qq, r)
// with qq ascending: every output sums its terms in one fixed sequential order, whatever
// the tile shape, the chunking of the contraction or the number of columns.
#pragma once

#include "cplx.cuh"

namespace hm {

template <class T, int TR, int TC, int NT> struct Tile {
    T v[NT][TR][TC];
};

// Row stride of a staged coefficient block: a whole number of row tiles, made odd so that
// the staging stores of consecutive qq do not fall into one shared-memory bank.
__host__ __device__ __forceinline__ int stage_ldw(int no, int TR) { return ((no + TR - 1) / TR * TR) | 1; }

// Columns of a staged vector block: a whole number of column tiles.
__host__ __device__ __forceinline__ int stage_ldr(int nrhs, int TC) { return (nrhs + TC - 1) / TC * TC; }

// Shared-memory entries of one staged step of contraction length nc.
__host__ __device__ __forceinline__ int stage_need(int no, int nc, int nrhs, int TR, int TC)
{
    return nc * stage_ldw(no, TR) + nc * stage_ldr(nrhs, TC);
}

// Tile index -> first row and first column of its tile.  Each run of 32 indices (one warp)
// covers a patch of pr row tiles x pc column tiles (pc = 4, or fewer when the block has fewer
// column tiles; pr = 32 / pc), so a warp's lanes read pr distinct staged rows and pc distinct
// column groups per contraction step instead of up to 32 rows: half the shared-memory
// wavefronts of a column-major walk for a 54-row block (measured: 16-column sweeps 7% faster,
// 32-column groups 2%).  nct = ntiles / nrt column tiles.  Slots used: round_up(nrt, pr) x
// round_up(nct, pc), at most NT x blockDim for every shape this library instantiates
// (row-tile counts up to 32, 64 or 128, column-tile counts up to 4, 8 or 16).  ok is false for
// an index outside the block.
struct TileRC {
    int row0, c0;
    bool ok;
};
template <int TR, int TC> __device__ __forceinline__ TileRC tile_rc(int tile, int nrt, int ntiles)
{
    const int nct = ntiles / nrt;
    const int pc = nct >= 4 ? 4 : (nct >= 2 ? 2 : 1), pr = 32 / pc;
    const int npr = (nrt + pr - 1) / pr, p = tile >> 5, l = tile & 31;
    const int rt = (p % npr) * pr + l % pr, ct = (p / npr) * pc + l / pr;
    return TileRC{rt * TR, ct * TC, rt < nrt && ct < nct};
}

// acc = x (or 0) at the thread's tiles; x(row, r) = x[row * xr + r * xc] when x != nullptr
template <class T, int TR, int TC, int NT>
__device__ __forceinline__ void tile_load(Tile<T, TR, TC, NT> &acc, const T *x, int64_t xr, int64_t xc, int no,
                                          int nrhs, int nrt, int ntiles)
{
#pragma unroll
    for (int t = 0; t < NT; ++t) {
        const TileRC m = tile_rc<TR, TC>(threadIdx.x + t * blockDim.x, nrt, ntiles);
        const int row0 = m.row0, r0 = m.c0;
#pragma unroll
        for (int a = 0; a < TR; ++a)
#pragma unroll
            for (int c = 0; c < TC; ++c)
                acc.v[t][a][c] = (x && m.ok && row0 + a < no && r0 + c < nrhs)
                                     ? x[(row0 + a) * xr + (r0 + c) * xc]
                                     : czero(T());
    }
}

// y(row, r) = acc at y[row * yr + r * yc] for the valid outputs of the thread's tiles
template <class T, int TR, int TC, int NT>
__device__ __forceinline__ void tile_store(const Tile<T, TR, TC, NT> &acc, T *y, int64_t yr, int64_t yc, int no,
                                           int nrhs, int nrt, int ntiles)
{
#pragma unroll
    for (int t = 0; t < NT; ++t) {
        const TileRC m = tile_rc<TR, TC>(threadIdx.x + t * blockDim.x, nrt, ntiles);
        const int row0 = m.row0, r0 = m.c0;
#pragma unroll
        for (int a = 0; a < TR; ++a)
#pragma unroll
            for (int c = 0; c < TC; ++c)
                if (m.ok && row0 + a < no && r0 + c < nrhs) y[(row0 + a) * yr + (r0 + c) * yc] = acc.v[t][a][c];
    }
}

// One staged product step (see the file comment); SUB selects acc -= M Y, else acc += M Y.
// Reads rows below round_up(no, TR) <= ldw and columns below stage_ldr(nrhs, TC) of the
// staged blocks; the padding entries only reach outputs that are never stored.
template <bool SUB, class T, int TR, int TC, int NT>
__device__ __forceinline__ void tile_mac(Tile<T, TR, TC, NT> &acc, const T *Ws, int ldw, const T *Ys, int ysq, int ysr,
                                         int nc, int nrt, int ntiles)
{
#pragma unroll
    for (int t = 0; t < NT; ++t) {
        const TileRC m = tile_rc<TR, TC>(threadIdx.x + t * blockDim.x, nrt, ntiles);
        if (m.ok) {
            const T *wp = Ws + m.row0;
            const T *yp = Ys + m.c0 * ysr;
#pragma unroll 2
            for (int qq = 0; qq < nc; ++qq) {
                T w[TR], yv[TC];
#pragma unroll
                for (int a = 0; a < TR; ++a) w[a] = wp[qq * ldw + a];
#pragma unroll
                for (int c = 0; c < TC; ++c) yv[c] = yp[qq * ysq + c * ysr];
#pragma unroll
                for (int a = 0; a < TR; ++a)
#pragma unroll
                    for (int c = 0; c < TC; ++c)
                        acc.v[t][a][c] = SUB ? cfms(w[a], yv[c], acc.v[t][a][c]) : cfma(w[a], yv[c], acc.v[t][a][c]);
            }
        }
    }
}

// Staging copy dst(e) = src(e) for e < count over the CTA's threads, SB loads in flight per
// thread before their stores (a plain loop would wait for each load before the next).
template <int SB = 8, class Ld, class St> __device__ __forceinline__ void stage_copy(int count, Ld &&ld, St &&st)
{
    for (int e0 = threadIdx.x; e0 < count; e0 += SB * blockDim.x) {
        decltype(ld(0)) v[SB];
#pragma unroll
        for (int u = 0; u < SB; ++u) {
            const int e = e0 + u * blockDim.x;
            if (e < count) v[u] = ld(e);
        }
#pragma unroll
        for (int u = 0; u < SB; ++u) {
            const int e = e0 + u * blockDim.x;
            if (e < count) st(e, v[u]);
        }
    }
}

// Tile shape for a column count: (1, 1, 1) up to 4 columns, (2, 2, 1) up to 16, (2, 4, 2) up
// to 64 (complex FP32); with 256 threads every output tile of a 64-row block is covered.
// Dispatches f.template run<TR, TC, NT>(maxw) with maxw the widest count of the shape.
template <class T, class F> __host__ auto tile_dispatch(int nrhs, F &&f)
{
    if (nrhs <= 4) return f.template run<1, 1, 1>(4);
    if constexpr (sizeof(T) == 16) return f.template run<2, 2, 1>(16);
    else {
        if (nrhs <= 16) return f.template run<2, 2, 1>(16);
        return f.template run<2, 4, 2>(64);
    }
}

}  // namespace hm
