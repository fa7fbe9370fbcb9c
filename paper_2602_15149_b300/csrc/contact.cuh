// Contact between bodies (Algorithm 1 step 1, Algorithm 2 step 2; <contcoeff>, <restcoef> of Sec. 3.3).
//
// Bodies are the specimens of a context.  The paper takes its contact model from its host framework without
// stating it; the one built here is a linear spring-dashpot normal force between particles of different
// bodies closer than the contact distance dc (the particle spacing):
//   delta = dc - r,  n = (x_i - x_j) / r,  k = kc E* dc^(dim - 2),  1/E* = (1 - nu_i^2)/E_i + (1 - nu_j^2)/E_j,
//   m* = m_i m_j / (m_i + m_j),  e = (e_i + e_j) / 2,  zeta = -ln e / sqrt(pi^2 + ln^2 e),
//   F_i = (k delta - 2 zeta sqrt(k m*) (v_i - v_j).n) n.
// With friction coefficients per body (<kfric>), Coulomb friction regularised near rest by the critical
// damping of the normal spring, c_t = 2 sqrt(k m*): the force gains -min(mu max(f_n, 0), c_t |v_t|) v_t/|v_t|,
// v_t = v_ij - (v_ij.n) n the sliding velocity and mu = (mu_i + mu_j) / 2.
//
// The pairs are found every step in the current configuration (FP64 positions X0 + u) on a spatial hash
// of cells of size dc: count the particles per bucket, scan, fill the bucket lists, sort each list by
// particle index (so that every sum runs in one order), then each particle visits the 3^dim cells around
// its own and keeps the particles of other bodies whose cell is the visited one (buckets may be shared).
// All buffers are allocated with the context; the sequence is a fixed set of launches, so it is captured
// in the step graph with the rest of the step.
#pragma once
#include "common.cuh"

namespace tl {

constexpr int kHashScanBlock = 1024;

__device__ __forceinline__ void contact_cell(const double *X0d, const double *u64, int n, int i, int dim, double dc,
                                             double x[3], int64_t c[3]) {
#pragma unroll
    for (int q = 0; q < 3; q++) {
        x[q] = q < dim ? X0d[q * n + i] + u64[q * n + i] : 0.0;
        c[q] = q < dim ? (int64_t)floor(x[q] / dc) : 0;
    }
}

// Spatial hash of a cell (large primes, xor), reduced to the table size (a power of two).
__device__ __forceinline__ int cell_hash(const int64_t c[3], int tsize) {
    const uint64_t h = ((uint64_t)c[0] * 73856093ull) ^ ((uint64_t)c[1] * 19349663ull) ^ ((uint64_t)c[2] * 83492791ull);
    return (int)(h & (uint64_t)(tsize - 1));
}

// Each particle's cell (kept for the pair search) and its place in its bucket.
template <typename T>
__global__ void __launch_bounds__(128) k_contact_count(StepArgs<T> a, const double *X0d, int dim, double dc, int tsize,
                                                       int *hcount, int *hbucket, int *hslot, int4 *hcell) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    double x[3];
    int64_t c[3];
    contact_cell(X0d, a.u64, a.n, i, dim, dc, x, c);
    const int b = cell_hash(c, tsize);
    hbucket[i] = b;
    hcell[i] = make_int4((int)c[0], (int)c[1], (int)c[2], 0);
    hslot[i] = atomicAdd(&hcount[b], 1);
}

// Exclusive scan of m ints in three launches with a fixed workspace: per-block scans and block sums,
// one block over the block sums (at most kHashScanBlock of them, 4 per thread), and the offsets.
__global__ void __launch_bounds__(kHashScanBlock) k_hscan_blocks(int m, const int *in, int *out, int *bsum) {
    __shared__ int sh[kHashScanBlock];
    const int i = blockIdx.x * kHashScanBlock + threadIdx.x;
    const int v = i < m ? in[i] : 0;
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < kHashScanBlock; o <<= 1) {
        const int t = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
        __syncthreads();
        sh[threadIdx.x] += t;
        __syncthreads();
    }
    if (i < m) out[i] = sh[threadIdx.x] - v;
    if (threadIdx.x == kHashScanBlock - 1) bsum[blockIdx.x] = sh[threadIdx.x];
}
__global__ void __launch_bounds__(kHashScanBlock) k_hscan_sums(int nb, int *bsum) {
    __shared__ int sh[kHashScanBlock];
    int v[4], tot = 0;
#pragma unroll
    for (int q = 0; q < 4; q++) {
        const int k = threadIdx.x * 4 + q;
        v[q] = k < nb ? bsum[k] : 0;
        tot += v[q];
    }
    sh[threadIdx.x] = tot;
    __syncthreads();
    for (int o = 1; o < kHashScanBlock; o <<= 1) {
        const int t = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
        __syncthreads();
        sh[threadIdx.x] += t;
        __syncthreads();
    }
    int run = sh[threadIdx.x] - tot;
#pragma unroll
    for (int q = 0; q < 4; q++) {
        const int k = threadIdx.x * 4 + q;
        if (k < nb) bsum[k] = run;
        run += v[q];
    }
}
__global__ void __launch_bounds__(kHashScanBlock) k_hscan_add(int m, int *out, const int *bsum) {
    const int i = blockIdx.x * kHashScanBlock + threadIdx.x;
    if (i < m) out[i] += bsum[blockIdx.x];
}

__global__ void k_contact_fill(int n, const int *hbucket, const int *hslot, const int *hstart, int *hlist) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) hlist[hstart[hbucket[i]] + hslot[i]] = i;
}

// Each bucket's list in ascending particle order (insertion sort; buckets hold a few particles).
__global__ void k_contact_sort(int tsize, const int *hcount, const int *hstart, int *hlist) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= tsize) return;
    const int m = hcount[b];
    if (m < 2) return;
    int *L = hlist + hstart[b];
    for (int p = 1; p < m; p++) {
        const int v = L[p];
        int q = p - 1;
        while (q >= 0 && L[q] > v) {
            L[q + 1] = L[q];
            q--;
        }
        L[q + 1] = v;
    }
}

// Contact acceleration of every particle from the current u and v (the step's level).
template <typename T, int DIM>
__global__ void __launch_bounds__(128) k_contact(StepArgs<T> a, const double *X0d, double dc, double kc,
                                                 const double *rest, const double *kfric, int tsize, const int *hcount,
                                                 const int *hstart, const int *hlist, const int4 *hcell, T *accc) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const int n = a.n;
    double xi[3];
#pragma unroll
    for (int k = 0; k < 3; k++) xi[k] = k < DIM ? X0d[k * n + i] + a.u64[k * n + i] : 0.0;
    const int4 own = hcell[i];  // the cells the particles were filed under
    const int64_t ci[3] = {own.x, own.y, own.z};
    const int si = a.spec[i];
    const double dt = a.dt[si];  // bodies in contact share one clock
    const MatT<T> mi = a.mats[a.mid[i]];
    const V4<T> Xi = a.X0V[i];
    const double massi = DIM == 3 ? (double)mi.rho * (double)Xi.w : (double)Xi.w;
    const V4<T> vri = a.vs_cur[i];
    const double vi[3] = {(double)vri.x, (double)vri.y, (double)vri.z};
    const double kdim = DIM == 3 ? kc * dc : kc;
    double acc[3] = {0.0, 0.0, 0.0};
    for (int dz = (DIM == 3 ? -1 : 0); dz <= (DIM == 3 ? 1 : 0); dz++)
        for (int dy = -1; dy <= 1; dy++)
            for (int dx = -1; dx <= 1; dx++) {
                const int64_t cc[3] = {ci[0] + dx, ci[1] + dy, ci[2] + dz};
                const int b = cell_hash(cc, tsize);
                const int beg = hstart[b], end = beg + hcount[b];
                for (int q = beg; q < end; q++) {
                    const int j = hlist[q];
                    if (a.spec[j] == si) continue;
                    const int4 cj = hcell[j];
                    if (cj.x != cc[0] || cj.y != cc[1] || cj.z != cc[2]) continue;  // another cell, same bucket
                    double xj[3];
#pragma unroll
                    for (int k = 0; k < 3; k++) xj[k] = k < DIM ? X0d[k * n + j] + a.u64[k * n + j] : 0.0;
                    double d[3], r2 = 0.0;
#pragma unroll
                    for (int k = 0; k < 3; k++) {
                        d[k] = xi[k] - xj[k];
                        r2 += d[k] * d[k];
                    }
                    if (!(r2 < dc * dc) || r2 == 0.0) continue;
                    const MatT<T> mj = a.mats[a.mid[j]];
                    const V4<T> Xj = a.X0V[j];
                    const double massj = DIM == 3 ? (double)mj.rho * (double)Xj.w : (double)Xj.w;
                    const V4<T> vrj = a.vs_cur[j];
                    const double vj[3] = {(double)vrj.x, (double)vrj.y, (double)vrj.z};
                    const double r = sqrt(r2);
                    const double kn = kdim / ((double)mi.cinv + (double)mj.cinv);
                    const double ms = massi * massj / (massi + massj);
                    const double e = 0.5 * (rest[si] + rest[a.spec[j]]);
                    double zeta = 0.0;
                    if (e < 1.0) {
                        const double le = log(e);
                        zeta = -le / sqrt(9.869604401089358 + le * le);  // pi^2
                    }
                    double vn = 0.0;
#pragma unroll
                    for (int k = 0; k < DIM; k++) vn += (vi[k] - vj[k]) * d[k] / r;
                    const double f = kn * (dc - r) - 2.0 * zeta * sqrt(kn * ms) * vn;
                    double F[3];
#pragma unroll
                    for (int k = 0; k < DIM; k++) F[k] = f * d[k] / r;
                    const double mu = kfric ? 0.5 * (kfric[si] + kfric[a.spec[j]]) : 0.0;
                    if (mu > 0.0 && f > 0.0) {  // friction (only while the pair is pressed together)
                        double vt[3], vt2 = 0.0;
#pragma unroll
                        for (int k = 0; k < DIM; k++) {
                            vt[k] = (vi[k] - vj[k]) - vn * d[k] / r;
                            vt2 += vt[k] * vt[k];
                        }
                        if (vt2 > 0.0) {
                            const double vtm = sqrt(vt2);
                            // Coulomb, regularised near rest, and at most stopping the sliding in one step
                            const double ft = fmin(fmin(mu * f, 2.0 * sqrt(kn * ms) * vtm), ms * vtm / dt);
#pragma unroll
                            for (int k = 0; k < DIM; k++) F[k] -= ft * vt[k] / vtm;
                        }
                    }
#pragma unroll
                    for (int k = 0; k < DIM; k++) acc[k] += F[k] / massi;
                }
            }
#pragma unroll
    for (int k = 0; k < DIM; k++) accc[k * n + i] = (T)acc[k];
}

}  // namespace tl
