// Shared device types of the TLSPH library.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "constitutive.cuh"

namespace tl {

template <typename T> struct alignas(4 * sizeof(T)) V4 { T x, y, z, w; };

__device__ __forceinline__ V4<float> ldg4(const V4<float> *p) {
    float4 f = __ldg(reinterpret_cast<const float4 *>(p));
    return V4<float>{f.x, f.y, f.z, f.w};
}
__device__ __forceinline__ V4<double> ldg4(const V4<double> *p) {
    const double2 *q = reinterpret_cast<const double2 *>(p);
    double2 a = __ldg(q), b = __ldg(q + 1);
    return V4<double>{a.x, a.y, b.x, b.y};
}

// Bulk prefetch of a contiguous global range into L2 by the TMA unit (one instruction,
// no registers).  ptr 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void prefetch_l2_bulk(const void *ptr, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(ptr), "r"(bytes) : "memory");
}

// Lane 0 of each warp prefetches the warp's SELL slice of neighbour indices (slices start
// on 128-byte boundaries and hold 32 x slice_len ints).
__device__ __forceinline__ void prefetch_slice(const int *col, const int64_t *slice_off, int i) {
    if ((threadIdx.x & 31) == 0) {
        const int64_t s = i >> 5;
        const int64_t b = slice_off[s], e = slice_off[s + 1];
        if (e > b) prefetch_l2_bulk(col + b, (uint32_t)((e - b) * sizeof(int)));
    }
}

// Boundary condition record (Sec. 3.3.2).
struct BCDev {
    int kind, comp_mask;
    double value[3];
    double t_start, t_end, ramp, area, inv_count;
    int expr[3];  // per component: index of a user-defined expression giving the value, or -1 (Sec. 3.3)
    int pad;
};
constexpr int kMaxBcPerParticle = 4;

// factor of a condition at time t: < 0 when inactive, else the ramp value in [0, 1]
__device__ __forceinline__ double bc_factor(const BCDev &b, double t) {
    if (t < b.t_start) return -1.0;
    if (b.t_end >= 0.0 && t > b.t_end) return -1.0;
    if (b.ramp > 0.0) {
        double f = (t - b.t_start) / b.ramp;
        return f < 1.0 ? f : 1.0;
    }
    return 1.0;
}

enum { kFlagNonfinite = 0, kFlagNoconv = 1, kFlagSingular = 2, kFlagRowOverflow = 3, kFlagTimeout = 4,
       kFlagCoincident = 5, kFlagBounds = 6, kNumFlags = 8 };

// All pointers of a step (device memory, cell-sorted order).
template <typename T> struct StepArgs {
    int n;
    const int64_t *slice_off;
    const int *row_len;
    const int *col;
    const unsigned *nmask;  // stencil layout: row masks, ceil(nsten / 32) arrays of n
    const int *soff;       // stencil differences j - i, ascending
    const int2 *runs;      // runs of consecutive differences: (first difference, first entry | length << 8)
    int nsten, nruns;      // stencil entries (0 = SELL-32 rows) and runs (the most of any table)
    int64_t halo;          // zero records before and after each gathered array (stencil layout)
    int sten_groups;       // stencil tables: 1, or one per specimen (kMaxStencil entries each)
    int lat_nx, lat_nxny;  // lattice walk (lattice.cuh): row and layer pitch, 0 = off
    int lat_cw;            // lattice walk: x width of a block's patch of rows (0 = whole rows, lattice.cuh)
    int lat_zc;            // lattice force pass streaming along z: planes per thread (0 = off)
    const unsigned *lmask; // lattice walk: one mask word per layer, 7 arrays of n
    const V4<T> *X0V;      // 3D (x, y, z, V0); 2D (x, y, V0, m0)
    const V4<T> *S1;       // sum_j V_j w_ij (X_j - X_i) / V_i (reference configuration)
    const V4<T> *ug_cur;   // gathered displacement copy (x, y, z, m0 in 3D)
    V4<T> *ug_next;
    const V4<T> *vs_cur;   // (vx, vy, vz, s)
    V4<T> *vs_next;
    V4<T> *Qa, *Qb;        // V_i P_i Ahat_i: 3D (q00 q01 q02 q10), (q11 q12 q20 q21); 2D Qa = (q00 q01 q10 q11)
    V4<T> *XQ;             // 3D pass-2 record of the stress pass: (x, y, z of X0V, V_i q22)
    T *G;                  // F - I from k_gradient, dim*dim arrays of n
    T *S3;                 // viscosity sum of pass 1a (without its factor h / rho_i), dim arrays of n
    T *Av;                 // viscous acceleration J F^-T Ahat S3 h / rho_i, dim arrays of n; null without viscosity
    T *LAP;                // phase-field Laplacian of pass 1a
    const T *Ahat;         // inverse of sum V w d d^T: 6 arrays of n (2D uses xx, yy, xy)
    T *K;                  // J2 state C_p^-1 - I, 6 arrays of n
    T *ep;                 // equivalent plastic strain
    T *H;                  // history functional
    T *sdot;               // phase-field rate
    double *u64;           // FP64 displacement, 3 arrays of n
    double *wext;          // work of the external forces on each particle since the start (FP64)
    const uint16_t *mid;
    const int *spec;
    const uint16_t *bcgrp;     // 0 = no condition, else group g -> grp_bcs[4 g .. 4 g + 3]
    const int16_t *grp_bcs;
    const BCDev *bcs;
    const MatT<T> *mats;
    double *t, *dt, *cmax;     // per specimen
    unsigned long long *vmax_bits, *amax_bits;  // per specimen, bits of a non-negative double
    double *last_vmax, *last_amax;
    unsigned int *done;
    int *flags;
    int nspec, dt_mode;
    double hd, cfl, fixed_dt;
    T h, inv2h, visc_eps;
    T grav[3];
    // Algorithm 2 (leapfrog): the step reads the half level through ug_cur / vs_cur, takes v_n from
    // v_own and writes v_{n+1}, u_{n+1} in place through vs_next / ug_next; acc_out keeps a_{n+1/2}
    int leap;
    const V4<T> *v_own;
    V4<T> *ug_half, *vs_half;  // predictor output
    // values of conditions given by expressions (Sec. 3.3), evaluated at the start of the step for the
    // particles in the expression list: expos[i] = list position p or -1; exval[(2 p + phase) * 12 +
    // 3 slot + k] and bit 3 slot + k of exskip[2 p + phase] (slot = the condition's place in the
    // particle's group, phase 1 = the Algorithm 2 predictor)
    const int *expos;
    const double *exval;
    const uint16_t *exskip;
    // contact accelerations between bodies of the step (null without contact), dim arrays of n
    const T *accc;
    // diagnostics (may be null)
    T *Fout, *Pout, *psi_out, *acc_out;
};

}  // namespace tl
