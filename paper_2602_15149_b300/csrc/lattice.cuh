// Lattice walk of the 3D step kernels: the neighbour loops of pass 1 and pass 2 for a particle set whose
// sorted order is a lattice order, with every pair difference j - i of the form
// dx + NX dy + NXNY dz over the ball dx^2 + dy^2 + dz^2 <= 9 (a lattice of spacing dp with R = 3 dp,
// jittered by less than the gap to the next lattice shell).  The ball has 122 entries besides its
// centre, in seven layers dz = -3..3 of 1, 21, 25, 29, 25, 21, 1 places; a row's mask holds one 32-bit
// word per layer (bit = the place in its layer, rows dy ascending, dx ascending; the centre keeps its
// place in layer 0 and its bit is never set).
//
// The walk reads no difference table and no index stream.  A thread takes P rows i, i + NX, ..,
// i + (P-1) NX (consecutive y rows of a lattice): the record at i + dx + NX y' + NXNY dz serves row p
// as its entry (dx, y' - p, dz), so a record is loaded once for up to P rows (the union of P shifted
// balls: 152 records for 244 pairs at P = 2, against 122 per row at P = 1).  Layers and the rows y' of
// a layer run as loops; a row of half width e in x runs as one of four straight-line bodies
// (e = 0..3) with immediate address offsets, so the code stays small enough for the instruction
// cache.  Each particle still visits its entries in ascending difference (layers dz ascending, rows
// ascending, dx ascending), which is the ascending column order of its CSR row: the walk adds the
// same terms in the same order as the stencil and SELL-32 walks, so all three give bit-identical steps.
#pragma once
#include "common.cuh"

namespace tl {

constexpr int kLatLayers = 7;  // dz = -3..3

// Half width in x of the ball's row (dy, dz): the largest e with e^2 <= 9 - dy^2 - dz^2, -1 if none.
__host__ __device__ constexpr int lat_ext(int dy, int dz) {
    const int r = 9 - dy * dy - dz * dz;
    if (r < 0) return -1;
    int e = 0;
    while ((e + 1) * (e + 1) <= r) e++;
    return e;
}
// Whether (dx, dy, dz) is an entry of the ball (the centre is not).
__host__ __device__ constexpr bool lat_entry(int dx, int dy, int dz) {
    const int e = lat_ext(dy, dz);
    return e >= 0 && dx >= -e && dx <= e && !(dx == 0 && dy == 0 && dz == 0);
}
// Place of (dx, dy, dz) in its layer's mask word (the same for dz and -dz).
__host__ __device__ constexpr int lat_bit(int dx, int dy, int dz) {
    const int M = lat_ext(0, dz);
    int b = 0;
    for (int y = -M; y < dy; y++) b += 2 * lat_ext(y, dz) + 1;
    return b + dx + lat_ext(dy, dz);
}
static_assert(lat_bit(3, 0, 0) == 17 && lat_bit(0, 3, 0) == 28 && lat_bit(0, 0, 3) == 0, "ball layout");
static_assert(lat_bit(2, 2, 1) == 24 && lat_bit(1, 2, 2) == 20, "ball layout");

// Row table of the ball, indexed [dz + 3][dy + 3]: half width in x (-1: no row), the place of the
// row's first entry in its layer word and the row's number of entries.
struct LatRows {
    signed char ext[7][7];
    unsigned char first[7][7];
    unsigned char width[7][7];  // entries of the row: 2 ext + 1, or 0 without a row
};
__host__ __device__ constexpr LatRows lat_rows_table() {
    LatRows t{};
    for (int dz = -3; dz <= 3; dz++)
        for (int dy = -3; dy <= 3; dy++) {
            const int e = lat_ext(dy, dz);
            t.ext[dz + 3][dy + 3] = (signed char)e;
            t.first[dz + 3][dy + 3] = (unsigned char)(e >= 0 ? lat_bit(-e, dy, dz) : 0);
            t.width[dz + 3][dy + 3] = (unsigned char)(e >= 0 ? 2 * e + 1 : 0);
        }
    return t;
}
__constant__ LatRows c_lat_rows = lat_rows_table();

// One row y' of a layer: the records rb + dx, dx = -EU..EU, each serving row p when abs(dx) <= e[p].
// bits[p] holds row p's mask bits aligned so that bit dx + EU belongs to entry dx.
template <int EU, int P, typename W>
__device__ __forceinline__ void lat_row(W &w, int rb, const int e[P], const unsigned bits[P]) {
#pragma unroll
    for (int k = 0; k <= 2 * EU; k++) {
        const int dx = k - EU;
        const int j = rb + dx;
        const auto rec = w.load(j);
#pragma unroll
        for (int p = 0; p < P; p++)
            if (P == 1 || (dx >= -e[p] && dx <= e[p])) w.pair(p, rec, j, ((bits[p] >> k) & 1u) != 0u);
    }
}

// Walk all seven layers for the thread's rows i0 + p NX (p < P).  W provides NX, NXNY, load(j) ->
// record and pair(p, record, j, on).  lmask: kLatLayers words of n per row; act[p]: whether row p is a
// particle (an inactive row has an empty mask).
template <int P, typename W> __device__ __forceinline__ void lat_walk(W &w, const unsigned *lmask, int n, int i0,
                                                                     const bool act[P]) {
#pragma unroll 1
    for (int L = 0; L < kLatLayers; L++) {
        unsigned lm[P];
#pragma unroll
        for (int p = 0; p < P; p++) lm[p] = act[p] ? __ldg(lmask + (int64_t)L * n + i0 + p * w.NX) : 0u;
        const int M = c_lat_rows.ext[L][3];
        const int base = i0 + (L - 3) * w.NXNY;
#pragma unroll 1
        for (int yp = -M; yp <= M + P - 1; yp++) {
            int e[P];
            unsigned bits[P];
            int EU = -1;
#pragma unroll
            for (int p = 0; p < P; p++) {
                const int dy = yp - p;
                e[p] = dy >= -M && dy <= M ? (int)c_lat_rows.ext[L][dy + 3] : -1;
                EU = e[p] > EU ? e[p] : EU;
            }
#pragma unroll
            for (int p = 0; p < P; p++) {
                const int dy = yp - p;
                bits[p] = e[p] >= 0 ? (lm[p] >> c_lat_rows.first[L][dy + 3]) << (EU - e[p]) : 0u;
            }
            const int rb = base + yp * w.NX;
            switch (EU) {
            case 0: lat_row<0, P>(w, rb, e, bits); break;
            case 1: lat_row<1, P>(w, rb, e, bits); break;
            case 2: lat_row<2, P>(w, rb, e, bits); break;
            default: lat_row<3, P>(w, rb, e, bits); break;
            }
        }
    }
}

// The walk of two rows with one pair body for both (W::pair2(record, j, on0, on1), e.g. in paired FP32
// arithmetic): a record outside one row's ball is computed for that row too, with its entry off.  The
// entries of each row are visited in the same order as by lat_walk.  (Splitting off the records only one
// row uses, at the x edges of a ball row, into one-row bodies measured slower: the edge loops cost more
// instructions than the packed bodies they save.)
template <int EU, typename W>
__device__ __forceinline__ void lat_row_pk(W &w, int rb, const int e[2], const unsigned bits[2]) {
#pragma unroll
    for (int k = 0; k <= 2 * EU; k++) {
        const int dx = k - EU;
        const int j = rb + dx;
        const auto rec = w.load(j);
        const bool on0 = dx >= -e[0] && dx <= e[0] && ((bits[0] >> k) & 1u) != 0u;
        const bool on1 = dx >= -e[1] && dx <= e[1] && ((bits[1] >> k) & 1u) != 0u;
        w.pair2(rec, j, on0, on1);
    }
}
template <typename W> __device__ __forceinline__ void lat_walk_pk(W &w, const unsigned *lmask, int n, int i0,
                                                                const bool act[2]) {
#pragma unroll 1
    for (int L = 0; L < kLatLayers; L++) {
        unsigned lm[2];
#pragma unroll
        for (int p = 0; p < 2; p++) lm[p] = act[p] ? __ldg(lmask + (int64_t)L * n + i0 + p * w.NX) : 0u;
        const int M = c_lat_rows.ext[L][3];
        const int base = i0 + (L - 3) * w.NXNY;
#pragma unroll 1
        for (int yp = -M; yp <= M + 1; yp++) {
            int e[2];
            unsigned bits[2];
            int EU = -1;
#pragma unroll
            for (int p = 0; p < 2; p++) {
                const int dy = yp - p;
                e[p] = dy >= -M && dy <= M ? (int)c_lat_rows.ext[L][dy + 3] : -1;
                EU = e[p] > EU ? e[p] : EU;
            }
#pragma unroll
            for (int p = 0; p < 2; p++) {
                const int dy = yp - p;
                bits[p] = e[p] >= 0 ? (lm[p] >> c_lat_rows.first[L][dy + 3]) << (EU - e[p]) : 0u;
            }
            const int rb = base + yp * w.NX;
            switch (EU) {
            case 0: lat_row_pk<0>(w, rb, e, bits); break;
            case 1: lat_row_pk<1>(w, rb, e, bits); break;
            case 2: lat_row_pk<2>(w, rb, e, bits); break;
            default: lat_row_pk<3>(w, rb, e, bits); break;
            }
        }
    }
}

// Rows of thread t: i0 = (t / NX) P NX + t % NX; threads = ceil(n / (P NX)) NX.
template <int P> __device__ __forceinline__ int lat_first_row(int t, int NX) {
    const int sr = t / NX;
    return sr * P * NX + (t - sr * NX);
}

// First row of thread tl of block b, and whether the thread owns rows.  The rows are cut into lines of
// NX (the rows i with the same i / NX: an x line of the lattice).
//   cw = 0: a block takes BS consecutive threads of lat_first_row (whole lines, P per thread group).
//   cw > 0 (a multiple of 32 that divides BS): a block takes a patch of cw consecutive x of BS / cw
//   groups of P consecutive lines; the blocks of a band of (BS / cw) P lines run along x first.  The
//   neighbour records of a patch (cw + 6 x, BS / cw P + 6 lines, 7 layers) are far fewer than those
//   of whole lines, so more of them stay in L1 while the block walks.  Threads past the end of a line
//   own nothing.  Either way every row i < n belongs to exactly one thread and one p.
template <int P, int BS>
__device__ __forceinline__ int lat_block_row(int b, int tl, int NX, int cw, bool &owns) {
    if (cw == 0) {
        owns = true;
        return lat_first_row<P>(b * BS + tl, NX);
    }
    const int chunks = (NX + cw - 1) / cw;
    const int band = b / chunks, g = tl / cw;
    const int x = (b - band * chunks) * cw + (tl - g * cw);
    owns = x < NX;
    return ((band * (BS / cw) + g) * P) * NX + x;
}

}  // namespace tl
