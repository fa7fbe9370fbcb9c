// Reference-configuration setup (runs once): cell keys, stable radix sort,
// neighbour lists, notch cut, correction tensors, SELL-32 neighbour layout.
//
// Neighbour predicate (Sec. 2.4): j != i, same specimen, r0^2 < R^2 with
// (two particles at the same reference position are an input error: the counting pass flags them)
// r0^2 = ((dx dx + dy dy) + dz dz) in FP64 round-to-nearest without fused
// multiply-add, so that the lists are bit-identical to any implementation
// that evaluates the same expression.
#pragma once
#include "common.cuh"

namespace tl {

// ---------------------------------------------------------------- bounding box
// One block; out[0..2] = min, out[3..5] = max over the first dim axes.
__global__ void k_bbox(int64_t n, int dim, const double *X /* n*3, orig order */, double *out) {
    __shared__ double smin[3][32], smax[3][32];
    double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x)
        for (int k = 0; k < dim; k++) {
            double x = X[3 * i + k];
            mn[k] = fmin(mn[k], x);
            mx[k] = fmax(mx[k], x);
        }
    for (int k = 0; k < 3; k++)
        for (int o = 16; o > 0; o >>= 1) {
            mn[k] = fmin(mn[k], __shfl_xor_sync(0xffffffffu, mn[k], o));
            mx[k] = fmax(mx[k], __shfl_xor_sync(0xffffffffu, mx[k], o));
        }
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0)
        for (int k = 0; k < 3; k++) { smin[k][w] = mn[k]; smax[k][w] = mx[k]; }
    __syncthreads();
    if (threadIdx.x == 0) {
        int nw = (blockDim.x + 31) >> 5;
        for (int k = 0; k < 3; k++) {
            double a = INFINITY, b = -INFINITY;
            for (int q = 0; q < nw; q++) { a = fmin(a, smin[k][q]); b = fmax(b, smax[k][q]); }
            if (k >= dim) { a = 0.0; b = 0.0; }
            out[k] = a;
            out[3 + k] = b;
        }
    }
}

// Cells of size R/3 centred on the planes X = Xmin + k R/3: coordinate
// floor((X - Xmin) / cs + 1/2); a pair with r0 < R is at most 3 cells apart per
// axis, and the search covers kCellRange = 4 to absorb rounding.  On a lattice of
// spacing R/3 every cell holds one particle, so the sorted order is lattice order.
constexpr int kCellRange = 4;
struct CellGrid {
    double xmin[3];
    double cs;          // cell size R / 3
    int64_t nc[3];      // cells per axis
    int dim;
};

__device__ __forceinline__ int64_t cell_coord(double x, double xmin, double cs) {
    return (int64_t)floor(__dadd_rn(__ddiv_rn(__dsub_rn(x, xmin), cs), 0.5));
}

// key = ((spec nz + cz) ny + cy) nx + cx
__global__ void k_cell_keys(int64_t n, CellGrid g, const double *X, const int *spec, unsigned long long *key,
                            int *id) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t c[3] = {0, 0, 0};
    for (int k = 0; k < g.dim; k++) c[k] = cell_coord(X[3 * i + k], g.xmin[k], g.cs);
    int64_t kk = (((int64_t)spec[i] * g.nc[2] + c[2]) * g.nc[1] + c[1]) * g.nc[0] + c[0];
    key[i] = (unsigned long long)kk;
    id[i] = (int)i;
}

// ---------------------------------------------------------------- stable LSD radix sort (8 bits / pass)
// One warp per block walks its tile in order; equal digits inside a 32-wide
// chunk are ranked with __match_any_sync, so every pass is stable.
constexpr int kSortTile = 4096;

__global__ void k_radix_hist(int64_t n, const unsigned long long *key, int shift, int64_t *hist /* 256 * nblk */) {
    __shared__ int cnt[256];
    for (int d = threadIdx.x; d < 256; d += blockDim.x) cnt[d] = 0;
    __syncwarp();
    int64_t b0 = (int64_t)blockIdx.x * kSortTile;
    int64_t b1 = min(n, b0 + kSortTile);
    for (int64_t i = b0 + threadIdx.x; i < b1; i += 32) atomicAdd(&cnt[(key[i] >> shift) & 255ull], 1);
    __syncwarp();
    for (int d = threadIdx.x; d < 256; d += 32) hist[(int64_t)d * gridDim.x + blockIdx.x] = cnt[d];
}

__global__ void k_radix_scatter(int64_t n, const unsigned long long *key, const int *val, int shift,
                                const int64_t *off /* scanned hist */, unsigned long long *key_out, int *val_out) {
    __shared__ int64_t base[256];
    for (int d = threadIdx.x; d < 256; d += 32) base[d] = off[(int64_t)d * gridDim.x + blockIdx.x];
    __syncwarp();
    int64_t b0 = (int64_t)blockIdx.x * kSortTile;
    int64_t b1 = min(n, b0 + kSortTile);
    const unsigned lt = (1u << threadIdx.x) - 1u;
    for (int64_t c0 = b0; c0 < b1; c0 += 32) {
        int64_t i = c0 + threadIdx.x;
        bool ok = i < b1;
        unsigned act = __ballot_sync(0xffffffffu, ok);
        int d = ok ? (int)((key[i] >> shift) & 255ull) : 256 + (int)threadIdx.x;
        unsigned peers = __match_any_sync(0xffffffffu, d) & act;
        int rank = __popc(peers & lt);
        int leader = __ffs(peers) - 1;
        int64_t pos = ok ? base[d] + rank : 0;
        if (ok) {
            key_out[pos] = key[i];
            val_out[pos] = val[i];
        }
        __syncwarp();
        if (ok && (int)threadIdx.x == leader) base[d] += __popc(peers);
        __syncwarp();
    }
}

// ---------------------------------------------------------------- exclusive scan (int64)
constexpr int kScanBlock = 1024;
__global__ void k_scan_block(int64_t m, const int64_t *in, int64_t *out, int64_t *bsum) {
    __shared__ int64_t ws[32];
    int64_t i = blockIdx.x * (int64_t)kScanBlock + threadIdx.x;
    int64_t v = i < m ? in[i] : 0;
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[w] = x;
    __syncthreads();
    if (w == 0) {
        int64_t s = ws[lane];
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        ws[lane] = s;
    }
    __syncthreads();
    int64_t pre = (w > 0 ? ws[w - 1] : 0) + x - v;
    if (i < m) out[i] = pre;
    if (threadIdx.x == kScanBlock - 1 && bsum) bsum[blockIdx.x] = ws[31];
}
__global__ void k_scan_add(int64_t m, int64_t *out, const int64_t *bscan) {
    int64_t i = blockIdx.x * (int64_t)kScanBlock + threadIdx.x;
    if (i < m && blockIdx.x > 0) out[i] += bscan[blockIdx.x];
}

// ---------------------------------------------------------------- neighbour search
struct NotchSet {
    const double *q;  // 12 per notch
    int count;
};

__device__ __forceinline__ double orient2(const double *a, const double *b, const double *p) {
    double t1 = __dmul_rn(__dsub_rn(b[0], a[0]), __dsub_rn(p[1], a[1]));
    double t2 = __dmul_rn(__dsub_rn(b[1], a[1]), __dsub_rn(p[0], a[0]));
    return __dsub_rn(t1, t2);
}
__device__ __forceinline__ double orient3(const double *a, const double *b, const double *c, const double *d) {
    double ux = __dsub_rn(b[0], a[0]), uy = __dsub_rn(b[1], a[1]), uz = __dsub_rn(b[2], a[2]);
    double vx = __dsub_rn(c[0], a[0]), vy = __dsub_rn(c[1], a[1]), vz = __dsub_rn(c[2], a[2]);
    double wx = __dsub_rn(d[0], a[0]), wy = __dsub_rn(d[1], a[1]), wz = __dsub_rn(d[2], a[2]);
    double c1 = __dsub_rn(__dmul_rn(vy, wz), __dmul_rn(vz, wy));
    double c2 = __dsub_rn(__dmul_rn(vz, wx), __dmul_rn(vx, wz));
    double c3 = __dsub_rn(__dmul_rn(vx, wy), __dmul_rn(vy, wx));
    return __dadd_rn(__dadd_rn(__dmul_rn(ux, c1), __dmul_rn(uy, c2)), __dmul_rn(uz, c3));
}
__device__ __forceinline__ bool opposite(double a, double b) { return (a > 0.0 && b < 0.0) || (a < 0.0 && b > 0.0); }

// Sec. 3.3.1 notch: bond P-Q (P from the lower caller id) crosses the notch inside it.
__device__ bool notch_cuts(const NotchSet &ns, int dim, const double *P, const double *Q) {
    const double margin = 1e-9;
    for (int k = 0; k < ns.count; k++) {
        const double *q = ns.q + 12 * k;
        if (dim == 2) {
            double A[2] = {q[0], q[1]}, B[2] = {q[3], q[4]};
            if (!opposite(orient2(A, B, P), orient2(A, B, Q))) continue;
            double o3 = orient2(P, Q, A), o4 = orient2(P, Q, B);
            if (!opposite(o3, o4)) continue;
            double t = __ddiv_rn(o3, __dsub_rn(o3, o4));
            if (t > margin && t < 1.0 - margin) return true;
        } else {
            const double *p1 = q, *p2 = q + 3, *p3 = q + 6, *p4 = q + 9;
            if (!opposite(orient3(p1, p2, p3, P), orient3(p1, p2, p3, Q))) continue;
            double e1 = orient3(P, Q, p1, p2), e2 = orient3(P, Q, p2, p3);
            double e3 = orient3(P, Q, p3, p4), e4 = orient3(P, Q, p4, p1);
            bool pos = e1 > 0.0 && e2 > 0.0 && e3 > 0.0 && e4 > 0.0;
            bool neg = e1 < 0.0 && e2 < 0.0 && e3 < 0.0 && e4 < 0.0;
            if (!pos && !neg) continue;
            double sum = __dadd_rn(__dadd_rn(__dadd_rn(e1, e2), e3), e4);
            if (__ddiv_rn(e1, sum) > margin && __ddiv_rn(e2, sum) > margin && __ddiv_rn(e3, sum) > margin &&
                __ddiv_rn(e4, sum) > margin)
                return true;
        }
    }
    return false;
}

__device__ __forceinline__ int64_t lower_bound_u64(const unsigned long long *a, int64_t n, unsigned long long v) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (a[mid] < v) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Count (FILL = false) or write (FILL = true) the neighbours of every sorted particle,
// visiting candidate cells in increasing key order so rows ascend by sorted index.
template <bool FILL>
__global__ void k_neighbours(int64_t n, CellGrid g, double R2, const unsigned long long *skey, const double *Xs /* 3 arrays */,
                             const int *sid /* caller id of sorted k */, NotchSet ns, int *row_len, const int64_t *row_ptr,
                             int *col, int *flags) {
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n) return;
    const double xi = Xs[k], yi = Xs[n + k], zi = Xs[2 * n + k];
    unsigned long long key = skey[k];
    int64_t cx = (int64_t)(key % (unsigned long long)g.nc[0]);
    unsigned long long r = key / (unsigned long long)g.nc[0];
    int64_t cy = (int64_t)(r % (unsigned long long)g.nc[1]);
    r /= (unsigned long long)g.nc[1];
    int64_t cz = (int64_t)(r % (unsigned long long)g.nc[2]);
    int64_t sp = (int64_t)(r / (unsigned long long)g.nc[2]);
    int cnt = 0;
    int64_t out = FILL ? row_ptr[k] : 0;
    const int dz0 = g.dim == 3 ? -kCellRange : 0, dz1 = g.dim == 3 ? kCellRange : 0;
    for (int dz = dz0; dz <= dz1; dz++) {
        int64_t z = cz + dz;
        if (z < 0 || z >= g.nc[2]) continue;
        for (int dy = -kCellRange; dy <= kCellRange; dy++) {
            int64_t y = cy + dy;
            if (y < 0 || y >= g.nc[1]) continue;
            int64_t x0 = max(cx - kCellRange, (int64_t)0), x1 = min(cx + kCellRange, g.nc[0] - 1);
            unsigned long long kb = (unsigned long long)((((sp * g.nc[2] + z) * g.nc[1] + y) * g.nc[0]) + x0);
            unsigned long long ke = kb + (unsigned long long)(x1 - x0 + 1);
            int64_t lo = lower_bound_u64(skey, n, kb), hi = lower_bound_u64(skey, n, ke);
            for (int64_t j = lo; j < hi; j++) {
                if (j == k) continue;
                double dx = __dsub_rn(Xs[j], xi), dy2 = __dsub_rn(Xs[n + j], yi);
                double r2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy2, dy2));
                if (g.dim == 3) {
                    double dz2 = __dsub_rn(Xs[2 * n + j], zi);
                    r2 = __dadd_rn(r2, __dmul_rn(dz2, dz2));
                }
                if (!(r2 < R2)) continue;
                if (!FILL && r2 == 0.0) atomicAdd(&flags[kFlagCoincident], 1);  // two particles at one place
                if (ns.count) {
                    int64_t a = sid[k] < sid[j] ? k : j, b = sid[k] < sid[j] ? j : k;
                    double P[3] = {Xs[a], Xs[n + a], Xs[2 * n + a]};
                    double Q[3] = {Xs[b], Xs[n + b], Xs[2 * n + b]};
                    if (notch_cuts(ns, g.dim, P, Q)) continue;
                }
                if (FILL) col[out++] = (int)j;
                cnt++;
            }
        }
    }
    if (!FILL) row_len[k] = cnt;
}

__global__ void k_widen_rows(int64_t n, const int *row_len, int64_t *len64, int *maxrow) {
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n) return;
    len64[k] = row_len[k];
    atomicMax(maxrow, row_len[k]);
}

// ---------------------------------------------------------------- correction tensor
// Ahat_i = (sum_j V_j w_ij d d^T)^-1, w = (1 - q/2)^3, d = X_j - X_i: the corrected
// kernel gradient of Sec. 2.4 is L_i gradW_ij = w_ij Ahat_i d (the Wendland constant
// alpha_D and the factor -5/h^2 cancel between L_i and gradW).  Positions are the
// values the step kernels use (rounded to T), so that the first-order consistency
// sum_j V_j (X_j - X_i) (x) L_i gradW_ij = I holds for the step's own geometry.
template <typename T>
__global__ void k_correction(int64_t n, int dim, const int64_t *row_ptr, const int *col, const V4<T> *X0V,
                             double inv2h, T *Ahat, int *flags) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    V4<T> xi = X0V[i];
    double M[6] = {0, 0, 0, 0, 0, 0};  // xx yy zz xy xz yz
    for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; e++) {
        V4<T> xj = X0V[col[e]];
        double d0 = (double)(xj.x - xi.x), d1 = (double)(xj.y - xi.y);
        double d2 = dim == 3 ? (double)(xj.z - xi.z) : 0.0;
        double V = dim == 3 ? (double)xj.w : (double)xj.z;
        double r = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
        double t = fmax(1.0 - r * inv2h, 0.0);
        double a = V * t * t * t;
        M[0] += a * d0 * d0;
        M[1] += a * d1 * d1;
        M[2] += a * d2 * d2;
        M[3] += a * d0 * d1;
        M[4] += a * d0 * d2;
        M[5] += a * d1 * d2;
    }
    double A[6] = {0, 0, 0, 0, 0, 0};
    bool bad;
    if (dim == 2) {
        double det = M[0] * M[1] - M[3] * M[3];
        double sc = fabs(M[0]) + fabs(M[1]);
        bad = !(fabs(det) > 1e-12 * sc * sc);
        A[0] = M[1] / det;
        A[1] = M[0] / det;
        A[3] = -M[3] / det;
    } else {
        double c00 = M[1] * M[2] - M[5] * M[5], c01 = M[4] * M[5] - M[3] * M[2], c02 = M[3] * M[5] - M[1] * M[4];
        double det = M[0] * c00 + M[3] * c01 + M[4] * c02;
        double sc = fabs(M[0]) + fabs(M[1]) + fabs(M[2]);
        bad = !(fabs(det) > 1e-12 * sc * sc * sc);
        A[0] = c00 / det;
        A[1] = (M[0] * M[2] - M[4] * M[4]) / det;
        A[2] = (M[0] * M[1] - M[3] * M[3]) / det;
        A[3] = c01 / det;
        A[4] = c02 / det;
        A[5] = (M[3] * M[4] - M[0] * M[5]) / det;
    }
    if (bad) atomicAdd(&flags[kFlagSingular], 1);
    for (int q = 0; q < 6; q++) Ahat[q * n + i] = bad ? T(0) : (T)A[q];
}

// ---------------------------------------------------------------- SELL-32 layout
// slice s = sorted particles [32 s, 32 s + 32); entry k of lane l at slice_off[s] + 32 k + l.
__global__ void k_slice_len(int64_t n, int64_t nslice, const int *row_len, int64_t *slen) {
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= nslice) return;
    int m = 0;
    for (int l = 0; l < 32; l++) {
        int64_t i = 32 * s + l;
        if (i < n) m = max(m, row_len[i]);
    }
    slen[s] = 32 * (int64_t)m;
}
__global__ void k_sell_fill(int64_t n, const int64_t *row_ptr, const int *col, const int64_t *slice_off, int *sell) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t base = slice_off[i >> 5] + (i & 31);
    int64_t b = row_ptr[i], e = row_ptr[i + 1];
    for (int64_t k = 0; k < e - b; k++) sell[base + 32 * k] = col[b + k];
}
__global__ void k_sell_pad(int64_t total, int *sell, int v) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < total) sell[i] = v;
}

// ---------------------------------------------------------------- stencil layout
// On a lattice in lattice order (one particle per fine cell, cells filling a box) the index
// difference j - i of a neighbour pair takes few distinct values: the lattice offsets within
// the support.  Per group of rows (a specimen: its own box, so its own row pitch), D = the sorted
// distinct differences; when every group has at most kMaxStencil of them, every row is a bit
// mask over its group's D (bit s set iff (i, i + D[s]) is a pair).  A row visits D in ascending
// order, which is the ascending column order of its CSR row: both layouts visit the same pairs in
// the same order.  The k-th visit of 32 consecutive rows of a group reads 32 consecutive particles.
constexpr int kMaxStencil = 128;
constexpr int kMaxRun = 8;  // longest run of consecutive differences the step kernels unroll

// Set bit (d + span) of group grp[i]'s bitmap (words_per_group words each) for every pair
// difference d of row i; *far counts pairs beyond +-span.  The bit is read first so that repeated
// differences cost no atomic.
__global__ void k_stencil_diffs(int64_t n, const int64_t *row_ptr, const int *col, const int *grp, int64_t span,
                                int64_t words_per_group, unsigned *bitmap, int *far) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    unsigned *bm = bitmap + (grp ? (int64_t)grp[i] : 0) * words_per_group;
    for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; k++) {
        const int64_t d = (int64_t)col[k] - i;
        if (d < -span || d >= span) {
            atomicAdd(far, 1);
            continue;
        }
        const uint64_t b = (uint64_t)(d + span);
        const unsigned bit = 1u << (b & 31);
        if (!(((volatile unsigned *)bm)[b >> 5] & bit)) atomicOr(&bm[b >> 5], bit);
    }
}

// Row masks over the row's group's D (D: kMaxStencil entries per group, nsten[g] used): words
// w = 0 .. nw - 1 at mask[w n + i].  A difference missing from D or a row out of ascending order
// counts in *bad.
__global__ void k_stencil_mask(int64_t n, const int64_t *row_ptr, const int *col, const int *grp, const int *D,
                               const int *nsten_g, int nw, unsigned *mask, int *bad) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int g = grp ? grp[i] : 0;
    const int *Dg = D + (int64_t)g * kMaxStencil;
    const int nsten = nsten_g[g];
    unsigned m0 = 0, m1 = 0, m2 = 0, m3 = 0;
    int s = 0;
    for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; k++) {
        const int64_t d = (int64_t)col[k] - i;
        while (s < nsten && (int64_t)Dg[s] < d) s++;
        if (s == nsten || (int64_t)Dg[s] != d) {
            atomicAdd(bad, 1);
            return;
        }
        const unsigned bit = 1u << (s & 31);
        switch (s >> 5) {
        case 0: m0 |= bit; break;
        case 1: m1 |= bit; break;
        case 2: m2 |= bit; break;
        default: m3 |= bit; break;
        }
        s++;  // strictly ascending rows: the next pair lies further on
    }
    mask[i] = m0;
    if (nw > 1) mask[n + i] = m1;
    if (nw > 2) mask[2 * n + i] = m2;
    if (nw > 3) mask[3 * n + i] = m3;
}

}  // namespace tl

namespace tl {
// Row masks of the lattice walk (lattice.cuh) from the stencil masks: stencil entry s of the table
// becomes bit map[s].y of layer word map[s].x.
__global__ void k_lattice_mask(int64_t n, int nsten, const unsigned *nmask, const int2 *map, unsigned *lmask) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    unsigned w[7] = {0u, 0u, 0u, 0u, 0u, 0u, 0u};
    for (int s = 0; s < nsten; s++) {
        if ((nmask[(int64_t)(s >> 5) * n + i] >> (s & 31)) & 1u) {
            const int2 m = map[s];
#pragma unroll
            for (int L = 0; L < 7; L++)
                if (m.x == L) w[L] |= 1u << m.y;
        }
    }
#pragma unroll
    for (int L = 0; L < 7; L++) lmask[(int64_t)L * n + i] = w[L];
}
}  // namespace tl
