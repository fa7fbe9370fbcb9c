// C-ABI of the TLSPH library (include/tlsph.h): context, device memory,
// reference setup and the step loop.  Every operation of the method runs in
// the kernels of setup_kernels.cuh and step_kernels.cuh; this file only
// allocates, copies, orders launches and reports status.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <type_traits>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/tlsph.h"
#include "expr_compile.h"
#include "contact.cuh"
#include "setup_kernels.cuh"
#include "step_kernels.cuh"

using namespace tl;

namespace {

constexpr int kThreads = 128;
inline unsigned blocks_for(int64_t n, int t = kThreads) { return (unsigned)((n + t - 1) / t); }

struct BCHost {
    int kind, comp_mask;
    double value[3];
    double t_start, t_end, ramp, area;
    std::vector<int64_t> ids;  // the masked particles (kept as a list: a batch has one condition per specimen)
    int64_t count;
    int expr[3] = {-1, -1, -1};  // user-defined expressions giving the components (Sec. 3.3)
};

}  // namespace

struct tlsph_ctx {
    tlsph_params p{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::string err;
    std::vector<tlsph_material> mats;
    int64_t n = 0;
    int nspec = 1;
    std::vector<double> X0h;  // n * 3, caller order
    std::vector<double> volh, v0h;
    std::vector<int32_t> midh, spech;
    std::vector<BCHost> bcs;
    std::vector<double> notches;
    bool built = false;
    int parity = 0;
    int64_t steps = 0, launches = 0, nnz = 0;
    int max_row = 0;
    int64_t nslice = 0, sell_total = 0;
    bool has_j2 = false, has_frac = false, has_visc = false;
    bool leap = false;  // Algorithm 2 (leapfrog) instead of Algorithm 1
    bool record_acc = false;
    size_t mem_limit = 0, mem_used = 0;  // cap on the context's state allocations (0 = none), and their total
    std::vector<size_t> alloc_bytes;     // size of each entry of allocs
    double bytes_per_step = 0.0;
    // device memory
    std::vector<void *> allocs;
    double *X0d = nullptr;  // sorted FP64 reference positions, 3 arrays
    int *perm = nullptr;    // sorted k -> caller id
    int64_t *row_ptr = nullptr;
    int *col = nullptr, *row_len = nullptr, *sell = nullptr;
    int64_t *slice_off = nullptr;
    int nsten = 0;                // stencil layout entries (0 = none)
    int *soff = nullptr;          // stencil differences j - i, ascending
    int2 *runs = nullptr;         // runs of consecutive differences
    int nruns = 0;
    int sten_groups = 1;          // stencil tables (one per specimen)
    int64_t halo = 0;             // zero elements before and after each gathered array (stencil layout)
    unsigned *nmask = nullptr;    // row masks over the stencil
    int lat_nx = 0, lat_nxny = 0; // lattice walk (3D FP32 lattices): row and layer pitch, 0 = none
    unsigned *lmask = nullptr;    // lattice walk: one mask word per layer, 7 arrays of n
    int lat_rows_grad = 1, lat_rows_force = 2;  // rows per thread of the two lattice kernels
    int lat_cw = 0;               // lattice kernels: x width of a block's patch of rows, 0 = whole rows
    int lat_zc = 0;               // lattice force pass streaming along z: planes per thread, 0 = off
    bool fuse_stress = false;     // the stress runs in the tail of the deformation-gradient kernel
    int layout = TLSPH_LAYOUT_AUTO;
    void *S1 = nullptr;  // sum_j V_j w_ij (X_j - X_i)
    void *X0V = nullptr, *ug[2] = {nullptr, nullptr}, *vs[2] = {nullptr, nullptr};
    void *S3 = nullptr, *Av = nullptr, *LAP = nullptr;  // viscosity sum, viscous acceleration, Laplacian
    void *Qa = nullptr, *Qb = nullptr, *XQ = nullptr, *G = nullptr;
    void *Ahat = nullptr, *K = nullptr, *ep = nullptr, *H = nullptr, *sdot = nullptr;
    double *u64 = nullptr;
    double *wext = nullptr;  // work of the external forces per particle (FP64)
    uint16_t *mid = nullptr, *bcgrp = nullptr;
    int *spec = nullptr;
    int16_t *grp_bcs = nullptr;
    BCDev *bcdev = nullptr;
    void *matsdev = nullptr;
    double *t = nullptr, *dt = nullptr, *cmax = nullptr, *last_v = nullptr, *last_a = nullptr;
    unsigned long long *vmax = nullptr, *amax = nullptr;
    unsigned int *done = nullptr;
    int *flags = nullptr;
    void *Fd = nullptr, *Pd = nullptr, *psid = nullptr, *accd = nullptr;
    double *energy = nullptr;
    int64_t flags_seen[kNumFlags] = {0};
    // learned constitutive surrogate attached to the context (FP32 steps only)
    bool sur_on = false;
    __nv_bfloat16 *sur_W = nullptr;
    float *sur_bias = nullptr, *sur_norm = nullptr;
    unsigned long long *sur_count = nullptr;  // network, outside the envelope, elastic trial
    int *sur_exact = nullptr;                 // list of the particles left to the exact update in a step
    unsigned *sur_nexact = nullptr;           // and its length
    int sur_tensor = TLSPH_TENSOR_TCGEN05;    // tensor path of the network pass
    int sur_scope = 0;
    // user-defined expressions (Sec. 3.3): compiled programs, their device tables (uploaded when the set
    // changes), and the particles whose boundary conditions use them (sorted order) with their values
    std::vector<ExProgram> exprogs;
    bool ex_dirty = false;
    ExInstr *excode = nullptr;
    double *exK = nullptr;
    ExProg *exprog = nullptr;
    int nexlist = 0;
    int *exlist = nullptr, *expos = nullptr;
    double *exval = nullptr;
    uint16_t *exskip = nullptr;
    // contact between bodies (the specimens): potential multiplier, contact distance, restitution per
    // body, spatial-hash tables and the contact accelerations of the step
    bool contact = false;
    double kc = 0.0;
    std::vector<double> resth;
    double *rest = nullptr;
    std::vector<double> kfrich;   // friction coefficient per body (empty = none)
    double *kfric = nullptr;
    int tsize = 0;
    int *hcount = nullptr, *hstart = nullptr, *hbucket = nullptr, *hslot = nullptr, *hlist = nullptr, *hbsum = nullptr;
    int4 *hcell = nullptr;
    void *accc = nullptr;
    // execution mode (TLSPH_MODE_*), block size, captured graph, persistent-launch barrier
    int mode = 0, bs = 128;
    int64_t graph_launches = 0;  // kernels in the captured two-step graph
    cudaGraphExec_t gexec = nullptr;
    unsigned int *bar = nullptr;
    bool barrier_test = false;
    // timing
    bool timing = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<int, int>> ev_pending;  // (kind, event index of start); stop = start + 1
    size_t ev_next = 0;
    double ms[3] = {0, 0, 0};
    int64_t cnt[3] = {0, 0, 0};
};

namespace {

tlsph_status fail(tlsph_ctx *c, tlsph_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    return st;
}

// An NVTX range over a C-ABI call, so that a timeline profiler shows the setup, each batch of steps and
// the autotuner by name (header-only NVTX; free when no tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

// Makes the context's device current for the duration of a call and restores the caller's.
struct DeviceScope {
    int prev = -1;
    explicit DeviceScope(int dev) {
        if (dev < 0) return;
        if (cudaGetDevice(&prev) != cudaSuccess) {
            cudaGetLastError();
            prev = -1;
            return;
        }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) cudaGetLastError();
    }
    ~DeviceScope() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

#define CK(call)                                                                                     \
    do {                                                                                             \
        cudaError_t e_ = (call);                                                                     \
        if (e_ != cudaSuccess) return fail(c, TLSPH_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)
#define CKL()                                                                                        \
    do {                                                                                             \
        c->launches++;                                                                               \
        cudaError_t e_ = cudaGetLastError();                                                         \
        if (e_ != cudaSuccess) return fail(c, TLSPH_ERR_CUDA, "launch: %s", cudaGetErrorString(e_)); \
    } while (0)

template <typename P> tlsph_status dalloc(tlsph_ctx *c, P **ptr, size_t bytes) {
    void *q = nullptr;
    if (bytes == 0) bytes = 16;
    if (c->mem_limit && c->mem_used + bytes > c->mem_limit)
        return fail(c, TLSPH_ERR_OOM, "device memory limit of %zu MiB reached (TLSPH_OPT_MEMORY_LIMIT)",
                    c->mem_limit >> 20);
    cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(c, TLSPH_ERR_OOM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
    }
    c->allocs.push_back(q);
    c->alloc_bytes.push_back(bytes);
    c->mem_used += bytes;
    *ptr = reinterpret_cast<P *>(q);
    return TLSPH_OK;
}
#define DA(ptr, bytes)                                  \
    do {                                                \
        tlsph_status s_ = dalloc(c, &(ptr), (bytes));   \
        if (s_ != TLSPH_OK) return s_;                  \
    } while (0)

void drop_graph(tlsph_ctx *c) {
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
}

void free_ex_tables(tlsph_ctx *c) {
    cudaFree(c->excode);
    cudaFree(c->exK);
    cudaFree(c->exprog);
    c->excode = nullptr;
    c->exK = nullptr;
    c->exprog = nullptr;
    c->ex_dirty = !c->exprogs.empty();
}

void free_device(tlsph_ctx *c) {
    drop_graph(c);
    for (void *q : c->allocs) cudaFree(q);
    c->allocs.clear();
    c->alloc_bytes.clear();
    c->mem_used = 0;
    c->rest = nullptr;
    c->kfric = nullptr;
    c->hcount = c->hstart = c->hbucket = c->hslot = c->hlist = c->hbsum = nullptr;
    c->hcell = nullptr;
    c->accc = nullptr;
    c->nexlist = 0;
    c->exlist = c->expos = nullptr;
    c->exval = nullptr;
    c->exskip = nullptr;
    c->X0d = nullptr;
    c->perm = nullptr;
    c->S1 = nullptr;
    c->nsten = 0;
    c->nruns = 0;
    c->sten_groups = 1;
    c->halo = 0;
    c->runs = nullptr;
    c->soff = nullptr;
    c->nmask = nullptr;
    c->lat_nx = c->lat_nxny = 0;
    c->lmask = nullptr;
    c->Fd = c->Pd = c->psid = c->accd = nullptr;
    c->bar = nullptr;
    c->sur_W = nullptr;
    c->sur_bias = c->sur_norm = nullptr;
    c->sur_count = nullptr;
    c->sur_exact = nullptr;
    c->sur_nexact = nullptr;
    c->sur_on = false;
    c->built = false;
}

void lame(const tlsph_material &m, double &lam, double &mu, double &kap) {
    lam = m.E * m.nu / ((1.0 + m.nu) * (1.0 - 2.0 * m.nu));
    mu = m.E / (2.0 * (1.0 + m.nu));
    kap = lam + 2.0 * mu / 3.0;
}
double sound_speed(const tlsph_material &m) {
    double lam, mu, kap;
    lame(m, lam, mu, kap);
    return sqrt((kap + 4.0 * mu / 3.0) / m.rho);
}

tlsph_status scan_exclusive(tlsph_ctx *c, int64_t m, const int64_t *in, int64_t *out) {
    // recursive block scan
    int64_t nb = (m + kScanBlock - 1) / kScanBlock;
    if (nb <= 1) {
        k_scan_block<<<1, kScanBlock, 0, c->stream>>>(m, in, out, nullptr);
        CKL();
        return TLSPH_OK;
    }
    int64_t *bs = nullptr, *bscan = nullptr;
    DA(bs, nb * sizeof(int64_t));
    DA(bscan, nb * sizeof(int64_t));
    k_scan_block<<<(unsigned)nb, kScanBlock, 0, c->stream>>>(m, in, out, bs);
    CKL();
    tlsph_status st = scan_exclusive(c, nb, bs, bscan);
    if (st != TLSPH_OK) return st;
    k_scan_add<<<(unsigned)nb, kScanBlock, 0, c->stream>>>(m, out, bscan);
    CKL();
    return TLSPH_OK;
}

template <typename T> __global__ void k_init_sorted(int64_t n, int dim, const int *perm, const double *X0c,
                                                    const double *volc, const double *v0c, const int *midc,
                                                    const int *specc, const uint16_t *grpc, const MatT<T> *mats,
                                                    double *X0d, V4<T> *vs, V4<T> *ug0, V4<T> *ug1, uint16_t *mid,
                                                    int *spec, uint16_t *bcgrp, int *first, int *last) {
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n) return;
    int64_t p = perm[k];
    for (int q = 0; q < 3; q++) X0d[q * n + k] = q < dim ? X0c[3 * p + q] : 0.0;
    const double V = volc[p];
    const int m = midc[p];
    double v[3] = {0, 0, 0};
    if (v0c)
        for (int q = 0; q < dim; q++) v[q] = v0c[dim * p + q];
    vs[k] = V4<T>{(T)v[0], (T)v[1], (T)v[2], T(1)};
    // gathered displacement starts at zero; in 3D its 4th slot carries the reference mass m0
    const T m0 = dim == 3 ? (T)((double)mats[m].rho * V) : T(0);
    ug0[k] = V4<T>{T(0), T(0), T(0), m0};
    ug1[k] = V4<T>{T(0), T(0), T(0), m0};
    mid[k] = (uint16_t)m;
    const int sp = specc ? specc[p] : 0;
    spec[k] = sp;
    bcgrp[k] = grpc[p];
    atomicMin(&first[sp], (int)k);
    atomicMax(&last[sp], (int)k);
}

// Reference positions in the step's precision, relative to an origin inside each specimen
// (the particle in the middle of its sorted range): small coordinates keep the relative
// precision of X_j - X_i in FP32, and a specimen gets the same values alone or in a batch.
template <typename T> __global__ void k_build_x0v(int64_t n, int dim, const double *X0d, const double *volc,
                                                  const int *perm, const int *spec, const int *first,
                                                  const int *last, const MatT<T> *mats, const uint16_t *mid,
                                                  V4<T> *X0V) {
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int sp = spec[k];
    const int64_t o = ((int64_t)first[sp] + (int64_t)last[sp]) / 2;
    T xs[3];
    for (int q = 0; q < 3; q++) xs[q] = (T)(X0d[q * n + k] - X0d[q * n + o]);
    const double V = volc[perm[k]];
    if (dim == 3) X0V[k] = V4<T>{xs[0], xs[1], xs[2], (T)V};
    else X0V[k] = V4<T>{xs[0], xs[1], (T)V, (T)((double)mats[mid[k]].rho * V)};
}

__global__ void k_fill_int(int64_t n, int *p, int v) {
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k < n) p[k] = v;
}

template <typename T> StepArgs<T> make_args(tlsph_ctx *c) {
    StepArgs<T> a{};
    const int cur = c->parity, nxt = c->parity ^ 1;
    a.n = (int)c->n;
    a.slice_off = c->slice_off;
    a.row_len = c->row_len;
    a.col = c->sell;
    const bool sten = c->layout != TLSPH_LAYOUT_CSR && c->nsten > 0;
    a.nsten = sten ? c->nsten : 0;
    a.nruns = sten ? c->nruns : 0;
    a.sten_groups = c->sten_groups;
    a.halo = c->halo;
    a.runs = sten ? c->runs : nullptr;
    a.soff = sten ? c->soff : nullptr;
    a.nmask = sten ? c->nmask : nullptr;
    const bool lat = c->layout == TLSPH_LAYOUT_AUTO && c->lat_nx > 0;
    a.lat_nx = lat ? c->lat_nx : 0;
    a.lat_nxny = lat ? c->lat_nxny : 0;
    a.lmask = lat ? c->lmask : nullptr;
    a.lat_cw = lat ? c->lat_cw : 0;
    a.lat_zc = lat ? c->lat_zc : 0;
    a.X0V = (const V4<T> *)c->X0V;
    a.S1 = (const V4<T> *)c->S1;
    a.ug_cur = (const V4<T> *)c->ug[cur];
    a.ug_next = (V4<T> *)c->ug[nxt];
    a.vs_cur = (const V4<T> *)c->vs[cur];
    a.vs_next = (V4<T> *)c->vs[nxt];
    a.Qa = (V4<T> *)c->Qa;
    a.Qb = (V4<T> *)c->Qb;
    a.XQ = (V4<T> *)c->XQ;
    a.G = (T *)c->G;
    a.S3 = (T *)c->S3;
    a.Av = c->has_visc ? (T *)c->Av : nullptr;
    a.LAP = (T *)c->LAP;
    a.Ahat = (const T *)c->Ahat;
    a.K = (T *)c->K;
    a.ep = (T *)c->ep;
    a.H = (T *)c->H;
    a.sdot = (T *)c->sdot;
    a.u64 = c->u64;
    a.wext = c->wext;
    a.mid = c->mid;
    a.spec = c->spec;
    a.bcgrp = c->bcgrp;
    a.grp_bcs = c->grp_bcs;
    a.bcs = c->bcdev;
    a.mats = (const MatT<T> *)c->matsdev;
    a.t = c->t;
    a.dt = c->dt;
    a.cmax = c->cmax;
    a.vmax_bits = c->vmax;
    a.amax_bits = c->amax;
    a.last_vmax = c->last_v;
    a.last_amax = c->last_a;
    a.done = c->done;
    a.flags = c->flags;
    a.nspec = c->nspec;
    a.dt_mode = c->p.dt_mode;
    a.hd = c->p.h;
    a.cfl = c->p.cfl;
    a.fixed_dt = c->p.fixed_dt;
    a.h = (T)c->p.h;
    a.inv2h = (T)(1.0 / (c->p.support * c->p.h));
    a.visc_eps = (T)(0.001 * c->p.h * c->p.h);
    for (int q = 0; q < 3; q++) a.grav[q] = (T)c->p.gravity[q];
    a.Fout = (T *)c->Fd;
    a.Pout = (T *)c->Pd;
    a.psi_out = (T *)c->psid;
    a.acc_out = c->record_acc ? (T *)c->accd : nullptr;
    a.expos = c->expos;
    a.exval = c->exval;
    a.exskip = c->exskip;
    a.accc = c->contact ? (const T *)c->accc : nullptr;
    return a;
}

// Uploads the compiled expressions (code, constants, offsets) when the set has changed.
tlsph_status ex_sync(tlsph_ctx *c) {
    if (!c->ex_dirty) return TLSPH_OK;
    drop_graph(c);  // a captured step refers to the old tables
    free_ex_tables(c);
    std::vector<ExInstr> code;
    std::vector<double> K;
    std::vector<ExProg> progs;
    for (const ExProgram &p : c->exprogs) {
        progs.push_back(ExProg{(int)code.size(), (int)p.code.size(), (int)K.size(), 0});
        code.insert(code.end(), p.code.begin(), p.code.end());
        K.insert(K.end(), p.consts.begin(), p.consts.end());
    }
    K.push_back(0.0);
    const size_t bc = code.size() * sizeof(ExInstr), bk = K.size() * sizeof(double), bp = progs.size() * sizeof(ExProg);
    if (cudaMalloc(&c->excode, bc) != cudaSuccess || cudaMalloc(&c->exK, bk) != cudaSuccess ||
        cudaMalloc(&c->exprog, bp) != cudaSuccess) {
        cudaGetLastError();
        free_ex_tables(c);
        return fail(c, TLSPH_ERR_OOM, "expression tables");
    }
    // synchronous copies: the host vectors end with this call
    if (cudaMemcpy(c->excode, code.data(), bc, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(c->exK, K.data(), bk, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(c->exprog, progs.data(), bp, cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        return fail(c, TLSPH_ERR_CUDA, "expression tables upload");
    }
    c->ex_dirty = false;
    return TLSPH_OK;
}

double ex_dx(const tlsph_ctx *c) { return c->p.dx > 0.0 ? c->p.dx : c->p.h / 1.5; }

// Arguments of the step kernels.  Algorithm 1 ping-pongs the displacement and velocity records
// (read cur, write next).  Algorithm 2 keeps them in place: the predictor writes the half level to
// the other buffers, the forces read it from there, and pass 2 writes v_{n+1}, u_{n+1} in place.
template <typename T> StepArgs<T> make_step_args(tlsph_ctx *c) {
    StepArgs<T> a = make_args<T>(c);
    if (c->leap) {
        const int cur = c->parity, nxt = c->parity ^ 1;
        a.leap = 1;
        a.v_own = (const V4<T> *)c->vs[cur];
        a.ug_half = (V4<T> *)c->ug[nxt];
        a.vs_half = (V4<T> *)c->vs[nxt];
        a.ug_cur = (const V4<T> *)c->ug[nxt];
        a.vs_cur = (const V4<T> *)c->vs[nxt];
        a.ug_next = (V4<T> *)c->ug[cur];
        a.vs_next = (V4<T> *)c->vs[cur];
        a.acc_out = (T *)c->accd;
    }
    return a;
}

// Algorithmic HBM bytes of one step: every particle's own records read / written once,
// neighbour gathers served on chip, neighbour indices read once per neighbour pass (4 B per
// pair, the CSR definition, whichever layout the kernels walk).
double algorithmic_bytes(const tlsph_ctx *c, size_t ts) {
    const int d = c->p.dim;
    const double n = (double)c->n, nnz = (double)c->nnz;
    const double v4 = 4.0 * ts, nsym = d == 3 ? 6 : 3, q = d * d * ts;
    const double vi = c->has_visc ? 1 : 0, fr = c->has_frac ? 1 : 0;
    // pass 1a: row, own X0V and u (and v, s for the viscosity or the Laplacian), Ahat; writes G, the
    // viscosity sum, the Laplacian
    const double grad = n * (4 + 8.0 / 32 + (2 + (vi + fr > 0 ? 1 : 0)) * v4 + nsym * ts + d * d * ts + vi * d * ts +
                             fr * ts) + 4.0 * nnz;
    // pass 1b: G, the viscosity sum, Ahat, material id, own X0V; writes V Q (3D with the position beside q22:
    // three float4) and the viscous acceleration
    double stress = n * (d * d * ts + nsym * ts + 2 + v4 + (d == 3 ? 3 * v4 : v4) + vi * 2 * d * ts);
    if (c->has_j2) stress += n * 2 * 7 * ts;
    if (c->has_frac) stress += n * (v4 + 2 * ts);
    // pass 2: row, own X0V, v and s, first moment, Q, viscous acceleration, ids, FP64 u read and
    // written, new u and v records; Laplacian, H and sdot with the phase field
    const double p2 = n * (4 + 8.0 / 32 + 3 * v4 + q + vi * d * ts + 2 + 4 + 2 + 2 * 8.0 * d + 2 * v4 + fr * 4 * ts) +
                      4.0 * nnz;
    return grad + stress + p2;
}

// Lattice walk (lattice.cuh) for a 3D stencil table whose differences all lie on the ball
// dx + NX dy + NXNY dz, dx^2 + dy^2 + dz^2 <= 9.  NX is found from the entry (-2, 1, 0), the smallest
// difference above 3; NXNY is the first difference above 3 NX + 3 under which every difference of the
// table falls on the ball (the entry (0, 0, 1)).  A table that is not such a lattice keeps the stencil
// walk.  The zero halo grows to the records the walk reads for up to four rows per thread.
tlsph_status build_lattice(tlsph_ctx *c, const int *D, int nst) {
    c->lat_nx = c->lat_nxny = 0;
    int d1 = -1;
    for (int s = 0; s < nst; s++)
        if (D[s] > 3) {
            d1 = D[s];
            break;
        }
    if (d1 < 0) return TLSPH_OK;
    const int64_t NX = (int64_t)d1 + 2;
    if (NX < 8) return TLSPH_OK;
    struct Pt { int dx, dy, dz; };
    std::vector<Pt> ball;
    for (int dz = -3; dz <= 3; dz++)
        for (int dy = -3; dy <= 3; dy++)
            for (int dx = -3; dx <= 3; dx++)
                if (lat_entry(dx, dy, dz)) ball.push_back(Pt{dx, dy, dz});
    std::vector<int2> map(nst);
    int64_t NXNY = 0;
    for (int s0 = 0; s0 < nst && NXNY == 0; s0++) {
        if (D[s0] <= 3 * NX + 3) continue;
        const int64_t cand = D[s0];
        if (cand < 7 * NX) continue;  // layers must not overlap
        bool all = true;
        for (int s = 0; s < nst && all; s++) {
            bool found = false;
            for (const Pt &q : ball)
                if (q.dx + NX * q.dy + cand * q.dz == (int64_t)D[s]) {
                    map[s] = make_int2(q.dz + 3, lat_bit(q.dx, q.dy, q.dz));
                    found = true;
                    break;
                }
            all = found;
        }
        if (all) NXNY = cand;
    }
    if (NXNY == 0 || NXNY > (int64_t)1 << 30) return TLSPH_OK;
    int64_t halo = c->halo;
    for (int p = 0; p < 4; p++)
        for (const Pt &q : ball) halo = std::max<int64_t>(halo, std::abs(q.dx + NX * (q.dy + p) + NXNY * q.dz));
    int2 *map_d;
    DA(map_d, nst * sizeof(int2));
    DA(c->lmask, (size_t)kLatLayers * c->n * sizeof(unsigned));
    CK(cudaMemcpyAsync(map_d, map.data(), nst * sizeof(int2), cudaMemcpyHostToDevice, c->stream));
    k_lattice_mask<<<blocks_for(c->n), kThreads, 0, c->stream>>>(c->n, nst, c->nmask, map_d, c->lmask);
    CKL();
    CK(cudaStreamSynchronize(c->stream));  // map is read before the host vector ends
    c->halo = halo;
    c->lat_nx = (int)NX;
    c->lat_nxny = (int)NXNY;
    return TLSPH_OK;
}

// Stencil layout of the CSR rows (lattice inputs), one table per specimen: the distinct pair
// differences j - i of the specimen's rows, kept when no specimen has more than kMaxStencil of
// them, and one bit mask per row.  Otherwise the context keeps the SELL-32 rows only.
tlsph_status build_stencil(tlsph_ctx *c) {
    const int64_t n = c->n;
    cudaStream_t s = c->stream;
    c->nsten = 0;
    if (n < 1 || c->nnz < 1) return TLSPH_OK;
    const int G = std::max(c->nspec, 1);
    // difference bitmaps: 2^25 bits in all, 2^14 .. 2^23 per specimen
    int64_t bits = (int64_t)1 << 23;
    while (bits > ((int64_t)1 << 14) && bits * G > ((int64_t)1 << 25)) bits >>= 1;
    const int64_t span = bits / 2, wpg = bits / 32;
    unsigned *bitmap;
    int *cnt;
    DA(bitmap, (size_t)G * wpg * sizeof(unsigned));
    DA(cnt, 2 * sizeof(int));
    CK(cudaMemsetAsync(bitmap, 0, (size_t)G * wpg * sizeof(unsigned), s));
    CK(cudaMemsetAsync(cnt, 0, 2 * sizeof(int), s));
    const int *grp = G > 1 ? c->spec : nullptr;
    k_stencil_diffs<<<blocks_for(n), kThreads, 0, s>>>(n, c->row_ptr, c->col, grp, span, wpg, bitmap, cnt);
    CKL();
    std::vector<unsigned> hb((size_t)G * wpg);
    int hc[2] = {0, 0};
    CK(cudaMemcpyAsync(hb.data(), bitmap, hb.size() * sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(hc, cnt, sizeof hc, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (hc[0] != 0) return TLSPH_OK;
    std::vector<int> D((size_t)G * kMaxStencil, 0), nst(G, 0);
    int nmax = 0;
    int64_t halo = 0;
    for (int g = 0; g < G; g++) {
        const unsigned *bm = hb.data() + (size_t)g * wpg;
        for (int64_t w = 0; w < wpg; w++)
            for (unsigned m = bm[w]; m; m &= m - 1) {
                if (nst[g] == kMaxStencil) return TLSPH_OK;
                const int d = (int)(32 * w + __builtin_ctz(m) - span);
                D[(size_t)g * kMaxStencil + nst[g]++] = d;
                halo = std::max<int64_t>(halo, std::abs((int64_t)d));
            }
        nmax = std::max(nmax, nst[g]);
    }
    if (nmax == 0) return TLSPH_OK;
    const int nw = (nmax + 31) / 32;
    int *nst_d;
    DA(c->soff, D.size() * sizeof(int));
    DA(nst_d, G * sizeof(int));
    DA(c->nmask, (size_t)nw * n * sizeof(unsigned));
    CK(cudaMemcpyAsync(c->soff, D.data(), D.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(nst_d, nst.data(), G * sizeof(int), cudaMemcpyHostToDevice, s));
    k_stencil_mask<<<blocks_for(n), kThreads, 0, s>>>(n, c->row_ptr, c->col, grp, c->soff, nst_d, nw, c->nmask,
                                                      cnt + 1);
    CKL();
    CK(cudaMemcpyAsync(hc, cnt, sizeof hc, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (hc[1] != 0) return TLSPH_OK;
    // runs of consecutive differences (at most kMaxRun long), kMaxStencil slots per specimen; unused
    // slots have length 0
    std::vector<int2> runs((size_t)G * kMaxStencil, make_int2(0, 0));
    int rmax = 0;
    for (int g = 0; g < G; g++) {
        const int *Dg = D.data() + (size_t)g * kMaxStencil;
        int r = 0;
        for (int a = 0; a < nst[g];) {
            int e = a + 1;
            while (e < nst[g] && Dg[e] == Dg[e - 1] + 1 && e - a < kMaxRun) e++;
            runs[(size_t)g * kMaxStencil + r++] = make_int2(Dg[a], a | ((e - a) << 8));
            a = e;
        }
        rmax = std::max(rmax, r);
    }
    DA(c->runs, runs.size() * sizeof(int2));
    CK(cudaMemcpyAsync(c->runs, runs.data(), runs.size() * sizeof(int2), cudaMemcpyHostToDevice, s));
    c->nruns = rmax;
    c->halo = halo;
    c->sten_groups = G;
    c->nsten = nmax;
    if (G == 1 && c->p.dim == 3 && c->p.precision == TLSPH_FP32_U64) return build_lattice(c, D.data(), nst[0]);
    return TLSPH_OK;
}

// Move a gathered array of n elements into a zero-filled allocation with c->halo elements
// before and after it (the stencil runs read every particle i + D, in range or not).
tlsph_status add_halo(tlsph_ctx *c, void *&ptr, size_t elem, int64_t n) {
    const int64_t H = c->halo;
    void *raw = nullptr;
    DA(raw, (size_t)(n + 2 * H) * elem);
    CK(cudaMemsetAsync(raw, 0, (size_t)(n + 2 * H) * elem, c->stream));
    void *np = (char *)raw + (size_t)H * elem;
    if (ptr) {
        CK(cudaMemcpyAsync(np, ptr, (size_t)n * elem, cudaMemcpyDeviceToDevice, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        auto it = std::find(c->allocs.begin(), c->allocs.end(), ptr);
        if (it != c->allocs.end()) {
            const size_t k = (size_t)(it - c->allocs.begin());
            cudaFree(*it);
            c->mem_used -= c->alloc_bytes[k];
            c->alloc_bytes.erase(c->alloc_bytes.begin() + (std::ptrdiff_t)k);
            c->allocs.erase(it);
        }
    }
    ptr = np;
    return TLSPH_OK;
}

template <typename T> tlsph_status build_impl(tlsph_ctx *c) {
    const int64_t n = c->n;
    const int dim = c->p.dim;
    free_device(c);
    cudaStream_t s = c->stream;
    // ---- inputs (caller order)
    double *X0c, *volc, *v0c = nullptr, *bbox;
    int *midc, *specc;
    uint16_t *grpc;
    DA(X0c, n * 3 * sizeof(double));
    DA(volc, n * sizeof(double));
    DA(midc, n * sizeof(int));
    DA(specc, n * sizeof(int));
    DA(grpc, n * sizeof(uint16_t));
    DA(bbox, 6 * sizeof(double));
    CK(cudaMemcpyAsync(X0c, c->X0h.data(), n * 3 * sizeof(double), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(volc, c->volh.data(), n * sizeof(double), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(midc, c->midh.data(), n * sizeof(int), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(specc, c->spech.data(), n * sizeof(int), cudaMemcpyHostToDevice, s));
    if (!c->v0h.empty()) {
        DA(v0c, n * dim * sizeof(double));
        CK(cudaMemcpyAsync(v0c, c->v0h.data(), n * dim * sizeof(double), cudaMemcpyHostToDevice, s));
    }
    // ---- boundary-condition groups
    std::vector<uint16_t> grph(n, 0);
    std::map<std::vector<int>, int> groups;
    std::vector<int16_t> grp_tab(4, -1);
    std::vector<std::vector<int>> per(n);
    for (size_t b = 0; b < c->bcs.size(); b++)
        for (int64_t pi : c->bcs[b].ids) per[pi].push_back((int)b);
    for (int64_t pi = 0; pi < n; pi++) {
        const std::vector<int> &ids = per[pi];
        if (ids.empty()) continue;
        if (ids.size() > (size_t)kMaxBcPerParticle)
            return fail(c, TLSPH_ERR_ARG, "particle %lld is covered by more than %d boundary conditions", (long long)pi,
                        kMaxBcPerParticle);
        auto it = groups.find(ids);
        int g;
        if (it == groups.end()) {
            g = (int)groups.size() + 1;
            if (g > 65535) return fail(c, TLSPH_ERR_ARG, "too many distinct boundary-condition groups");
            groups[ids] = g;
            for (int q = 0; q < 4; q++) grp_tab.push_back(q < (int)ids.size() ? (int16_t)ids[q] : (int16_t)-1);
        } else {
            g = it->second;
        }
        grph[pi] = (uint16_t)g;
    }
    CK(cudaMemcpyAsync(grpc, grph.data(), n * sizeof(uint16_t), cudaMemcpyHostToDevice, s));
    DA(c->grp_bcs, grp_tab.size() * sizeof(int16_t));
    CK(cudaMemcpyAsync(c->grp_bcs, grp_tab.data(), grp_tab.size() * sizeof(int16_t), cudaMemcpyHostToDevice, s));
    std::vector<BCDev> bch(std::max<size_t>(c->bcs.size(), 1));
    for (size_t b = 0; b < c->bcs.size(); b++) {
        const BCHost &h = c->bcs[b];
        BCDev &d = bch[b];
        d.kind = h.kind;
        d.comp_mask = h.comp_mask;
        for (int q = 0; q < 3; q++) d.value[q] = h.value[q];
        d.t_start = h.t_start;
        d.t_end = h.t_end;
        d.ramp = h.ramp;
        d.area = h.area;
        d.inv_count = h.count > 0 ? 1.0 / (double)h.count : 0.0;
        for (int q = 0; q < 3; q++) d.expr[q] = h.expr[q];
        d.pad = 0;
    }
    for (size_t b = c->bcs.size(); b < bch.size(); b++)
        for (int q = 0; q < 3; q++) bch[b].expr[q] = -1;
    DA(c->bcdev, bch.size() * sizeof(BCDev));
    CK(cudaMemcpyAsync(c->bcdev, bch.data(), bch.size() * sizeof(BCDev), cudaMemcpyHostToDevice, s));
    // ---- materials
    std::vector<MatT<T>> mt(c->mats.size());
    c->has_j2 = c->has_frac = c->has_visc = false;
    for (size_t k = 0; k < c->mats.size(); k++) {
        const tlsph_material &m = c->mats[k];
        double lam, mu, kap;
        lame(m, lam, mu, kap);
        MatT<T> &d = mt[k];
        d.model = m.model;
        d.fracture = (m.model != TLSPH_MODEL_J2 && m.fracture) ? 1 : 0;
        d.rho = (T)m.rho;
        d.mu = (T)mu;
        d.kappa = (T)kap;
        d.sy0 = (T)m.sigma_y0;
        d.Hh = (T)m.H_hard;
        d.beta1 = (T)m.beta1;
        d.beta2 = (T)m.beta2;
        d.c0 = (T)sound_speed(m);
        d.Gc = (T)m.Gc;
        d.eps0 = (T)m.eps0;
        d.s_lim = (T)m.s_lim;
        d.mass_scale = T(1);
        d.lam = (T)lam;
        d.cinv = (T)((1.0 - m.nu * m.nu) / m.E);
    }
    std::vector<char> used(c->mats.size(), 0);
    for (int64_t pi = 0; pi < n; pi++) used[c->midh[pi]] = 1;
    for (size_t k = 0; k < c->mats.size(); k++)
        if (used[k]) {
            if (c->mats[k].model == TLSPH_MODEL_J2) c->has_j2 = true;
            if (mt[k].fracture) c->has_frac = true;
            if (c->mats[k].beta1 != 0.0 || c->mats[k].beta2 != 0.0) c->has_visc = true;
        }
    DA(c->matsdev, mt.size() * sizeof(MatT<T>));
    CK(cudaMemcpyAsync(c->matsdev, mt.data(), mt.size() * sizeof(MatT<T>), cudaMemcpyHostToDevice, s));
    // ---- notches
    double *notchd = nullptr;
    int nn = (int)(c->notches.size() / 12);
    if (nn) {
        DA(notchd, c->notches.size() * sizeof(double));
        CK(cudaMemcpyAsync(notchd, c->notches.data(), c->notches.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    }
    // ---- cell grid (same formulas as the specification of the predicate)
    k_bbox<<<1, 1024, 0, s>>>(n, dim, X0c, bbox);
    CKL();
    double bb[6];
    CK(cudaMemcpyAsync(bb, bbox, sizeof bb, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const double R = c->p.support * c->p.h, R2 = R * R;
    CellGrid g;
    g.dim = dim;
    g.cs = R / 3.0;
    for (int k = 0; k < 3; k++) {
        g.xmin[k] = bb[k];
        g.nc[k] = (int64_t)floor((bb[3 + k] - bb[k]) / g.cs + 0.5) + 1;
    }
    double maxkey = ((double)c->nspec * g.nc[2] * g.nc[1] * g.nc[0]);
    if (!(maxkey < 9.0e18)) return fail(c, TLSPH_ERR_ARG, "cell grid too large");
    int bits = 1;
    while (bits < 64 && (double)(1ull << bits) < maxkey) bits++;
    // ---- keys and stable sort
    unsigned long long *key[2];
    int *val[2];
    DA(key[0], n * 8);
    DA(key[1], n * 8);
    DA(val[0], n * 4);
    DA(val[1], n * 4);
    k_cell_keys<<<blocks_for(n), kThreads, 0, s>>>(n, g, X0c, specc, key[0], val[0]);
    CKL();
    const int64_t nblk = (n + kSortTile - 1) / kSortTile;
    int64_t *hist, *hoff;
    DA(hist, 256 * nblk * sizeof(int64_t));
    DA(hoff, 256 * nblk * sizeof(int64_t));
    int cur = 0;
    for (int shift = 0; shift < bits; shift += 8) {
        k_radix_hist<<<(unsigned)nblk, 32, 0, s>>>(n, key[cur], shift, hist);
        CKL();
        tlsph_status st = scan_exclusive(c, 256 * nblk, hist, hoff);
        if (st != TLSPH_OK) return st;
        k_radix_scatter<<<(unsigned)nblk, 32, 0, s>>>(n, key[cur], val[cur], shift, hoff, key[cur ^ 1], val[cur ^ 1]);
        CKL();
        cur ^= 1;
    }
    c->perm = val[cur];
    unsigned long long *skey = key[cur];
    // ---- sorted particle arrays
    DA(c->X0d, 3 * n * sizeof(double));
    DA(c->X0V, n * sizeof(V4<T>));
    DA(c->vs[0], n * sizeof(V4<T>));
    DA(c->vs[1], n * sizeof(V4<T>));
    DA(c->ug[0], n * sizeof(V4<T>));
    DA(c->ug[1], n * sizeof(V4<T>));
    DA(c->mid, n * sizeof(uint16_t));
    DA(c->spec, n * sizeof(int));
    DA(c->bcgrp, n * sizeof(uint16_t));
    int *sfirst, *slast;
    DA(sfirst, c->nspec * sizeof(int));
    DA(slast, c->nspec * sizeof(int));
    k_fill_int<<<blocks_for(c->nspec), kThreads, 0, s>>>(c->nspec, sfirst, (int)n);
    CKL();
    k_fill_int<<<blocks_for(c->nspec), kThreads, 0, s>>>(c->nspec, slast, -1);
    CKL();
    k_init_sorted<T><<<blocks_for(n), kThreads, 0, s>>>(n, dim, c->perm, X0c, volc, v0c, midc, specc, grpc,
                                                        (const MatT<T> *)c->matsdev, c->X0d, (V4<T> *)c->vs[0],
                                                        (V4<T> *)c->ug[0], (V4<T> *)c->ug[1], c->mid, c->spec,
                                                        c->bcgrp, sfirst, slast);
    CKL();
    k_build_x0v<T><<<blocks_for(n), kThreads, 0, s>>>(n, dim, c->X0d, volc, c->perm, c->spec, sfirst, slast,
                                                      (const MatT<T> *)c->matsdev, c->mid, (V4<T> *)c->X0V);
    CKL();
    CK(cudaMemcpyAsync(c->vs[1], c->vs[0], n * sizeof(V4<T>), cudaMemcpyDeviceToDevice, s));
    // ---- particles whose boundary conditions use expressions (sorted order), and their value slots
    {
        std::vector<uint8_t> has_ex(n, 0);
        for (const BCHost &b : c->bcs)
            if (b.expr[0] >= 0 || b.expr[1] >= 0 || b.expr[2] >= 0)
                for (int64_t pi : b.ids) has_ex[pi] = 1;
        int64_t m = 0;
        for (int64_t pi = 0; pi < n; pi++) m += has_ex[pi];
        if (m > 0) {
            if (m > INT32_MAX / 24) return fail(c, TLSPH_ERR_ARG, "too many particles with expression conditions");
            std::vector<int> permh(n), list, pos(n, -1);
            CK(cudaMemcpyAsync(permh.data(), c->perm, n * sizeof(int), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            for (int64_t k = 0; k < n; k++)
                if (has_ex[permh[k]]) {
                    pos[k] = (int)list.size();
                    list.push_back((int)k);
                }
            c->nexlist = (int)m;
            DA(c->exlist, m * sizeof(int));
            DA(c->expos, n * sizeof(int));
            DA(c->exval, m * 24 * sizeof(double));
            DA(c->exskip, m * 2 * sizeof(uint16_t));
            CK(cudaMemcpyAsync(c->exlist, list.data(), m * sizeof(int), cudaMemcpyHostToDevice, s));
            CK(cudaMemcpyAsync(c->expos, pos.data(), n * sizeof(int), cudaMemcpyHostToDevice, s));
            CK(cudaMemsetAsync(c->exval, 0, m * 24 * sizeof(double), s));
            CK(cudaMemsetAsync(c->exskip, 0xff, m * 2 * sizeof(uint16_t), s));
            CK(cudaStreamSynchronize(s));  // the host vectors end with this block
            tlsph_status st = ex_sync(c);
            if (st != TLSPH_OK) return st;
        }
    }
    // ---- neighbours (count, scan, fill)
    DA(c->row_len, n * sizeof(int));
    DA(c->row_ptr, (n + 1) * sizeof(int64_t));
    NotchSet ns{notchd, nn};
    DA(c->flags, kNumFlags * sizeof(int));
    CK(cudaMemsetAsync(c->flags, 0, kNumFlags * sizeof(int), s));
    k_neighbours<false><<<blocks_for(n), kThreads, 0, s>>>(n, g, R2, skey, c->X0d, c->perm, ns, c->row_len, nullptr,
                                                           nullptr, c->flags);
    CKL();
    int64_t *len64;
    DA(len64, (n + 1) * sizeof(int64_t));
    int *maxrow;
    DA(maxrow, sizeof(int));
    CK(cudaMemsetAsync(maxrow, 0, sizeof(int), s));
    CK(cudaMemsetAsync(len64, 0, (n + 1) * sizeof(int64_t), s));
    k_widen_rows<<<blocks_for(n), kThreads, 0, s>>>(n, c->row_len, len64, maxrow);
    CKL();
    CK(cudaMemcpyAsync(&c->max_row, maxrow, sizeof(int), cudaMemcpyDeviceToHost, s));
    tlsph_status st = scan_exclusive(c, n + 1, len64, c->row_ptr);
    if (st != TLSPH_OK) return st;
    CK(cudaMemcpyAsync(&c->nnz, c->row_ptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (c->nnz >= (int64_t)1 << 31) return fail(c, TLSPH_ERR_ARG, "too many neighbour pairs for 32-bit indices");
    DA(c->col, std::max<int64_t>(c->nnz, 1) * sizeof(int));
    k_neighbours<true><<<blocks_for(n), kThreads, 0, s>>>(n, g, R2, skey, c->X0d, c->perm, ns, c->row_len, c->row_ptr,
                                                          c->col, c->flags);
    CKL();
    // ---- flags, correction tensors
        for (int q = 0; q < kNumFlags; q++) c->flags_seen[q] = 0;
    DA(c->Ahat, 6 * n * sizeof(T));
    k_correction<T><<<blocks_for(n), kThreads, 0, s>>>(n, dim, c->row_ptr, c->col, (const V4<T> *)c->X0V,
                                                       1.0 / R, (T *)c->Ahat, c->flags);
    CKL();
    // ---- SELL-32 layout
    c->nslice = (n + 31) / 32;
    int64_t *slen;
    DA(slen, (c->nslice + 1) * sizeof(int64_t));
    CK(cudaMemsetAsync(slen, 0, (c->nslice + 1) * sizeof(int64_t), s));
    k_slice_len<<<blocks_for(c->nslice), kThreads, 0, s>>>(n, c->nslice, c->row_len, slen);
    CKL();
    DA(c->slice_off, (c->nslice + 1) * sizeof(int64_t));
    st = scan_exclusive(c, c->nslice + 1, slen, c->slice_off);
    if (st != TLSPH_OK) return st;
    CK(cudaMemcpyAsync(&c->sell_total, c->slice_off + c->nslice, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    DA(c->sell, std::max<int64_t>(c->sell_total, 1) * sizeof(int));
    k_sell_pad<<<blocks_for(std::max<int64_t>(c->sell_total, 1)), kThreads, 0, s>>>(c->sell_total, c->sell, 0);
    CKL();
    k_sell_fill<<<blocks_for(n), kThreads, 0, s>>>(n, c->row_ptr, c->col, c->slice_off, c->sell);
    CKL();
    st = build_stencil(c);
    if (st != TLSPH_OK) return st;
    if (c->nsten > 0) {  // zero halo around the gathered arrays
        st = add_halo(c, c->X0V, sizeof(V4<T>), n);
        for (int q = 0; q < 2 && st == TLSPH_OK; q++) {
            st = add_halo(c, c->vs[q], sizeof(V4<T>), n);
            if (st == TLSPH_OK) st = add_halo(c, c->ug[q], sizeof(V4<T>), n);
        }
        if (st != TLSPH_OK) return st;
    }
    // ---- state
    DA(c->u64, 3 * n * sizeof(double));
    CK(cudaMemsetAsync(c->u64, 0, 3 * n * sizeof(double), s));
    DA(c->wext, n * sizeof(double));
    CK(cudaMemsetAsync(c->wext, 0, n * sizeof(double), s));
    if (c->nsten > 0) {
        c->Qa = c->Qb = c->XQ = nullptr;
        st = add_halo(c, c->Qa, sizeof(V4<T>), n);
        if (st == TLSPH_OK) st = add_halo(c, c->Qb, sizeof(V4<T>), dim == 3 ? n : 1);
        if (st == TLSPH_OK) st = add_halo(c, c->XQ, sizeof(V4<T>), dim == 3 ? n : 1);
        if (st != TLSPH_OK) return st;
    } else {
        DA(c->Qa, n * sizeof(V4<T>));
        DA(c->Qb, (dim == 3 ? n : 1) * sizeof(V4<T>));
        DA(c->XQ, (dim == 3 ? n : 1) * sizeof(V4<T>));
    }
    CK(cudaMemsetAsync(c->Qa, 0, n * sizeof(V4<T>), s));
    DA(c->G, dim * dim * n * sizeof(T));
    DA(c->S3, dim * n * sizeof(T));
    DA(c->Av, dim * n * sizeof(T));
    DA(c->LAP, n * sizeof(T));
    CK(cudaMemsetAsync(c->LAP, 0, n * sizeof(T), s));
    DA(c->K, 6 * n * sizeof(T));
    CK(cudaMemsetAsync(c->K, 0, 6 * n * sizeof(T), s));
    DA(c->ep, n * sizeof(T));
    CK(cudaMemsetAsync(c->ep, 0, n * sizeof(T), s));
    DA(c->H, n * sizeof(T));
    CK(cudaMemsetAsync(c->H, 0, n * sizeof(T), s));
    DA(c->sdot, n * sizeof(T));
    CK(cudaMemsetAsync(c->sdot, 0, n * sizeof(T), s));
    DA(c->accd, dim * n * sizeof(T));
    CK(cudaMemsetAsync(c->accd, 0, dim * n * sizeof(T), s));
    DA(c->energy, 8 * sizeof(double));
    // ---- per-specimen clocks (eq. dt_criterion)
    const int ns_ = c->nspec;
    std::vector<double> cm(ns_, 0.0), vm0(ns_, 0.0), t0(ns_, 0.0), dt0(ns_, 0.0);
    for (int64_t pi = 0; pi < n; pi++) {
        int sp = c->spech.empty() ? 0 : c->spech[pi];
        double cs = sound_speed(c->mats[c->midh[pi]]);
        if (cs > cm[sp]) cm[sp] = cs;
        double vv = 0.0;
        for (int k = 0; k < 3; k++) {
            double x = (!c->v0h.empty() && k < dim) ? c->v0h[dim * pi + k] : 0.0;
            vv += x * x;
        }
        vv = sqrt(vv);
        if (vv > vm0[sp]) vm0[sp] = vv;
    }
    if (c->contact) {  // bodies in contact share one clock: the largest sound speed of all
        double m = 0.0;
        for (int sp = 0; sp < ns_; sp++) m = std::max(m, cm[sp]);
        for (int sp = 0; sp < ns_; sp++) cm[sp] = m;
    }
    for (int sp = 0; sp < ns_; sp++) {
        const double h = c->p.h;
        if (c->p.dt_mode == TLSPH_DT_FIXED) dt0[sp] = c->p.fixed_dt;
        else if (c->p.dt_mode == TLSPH_DT_CFL_STATIC) dt0[sp] = c->p.cfl * h / cm[sp];
        else dt0[sp] = c->p.cfl * (h / (cm[sp] + vm0[sp]));
    }
    DA(c->t, ns_ * sizeof(double));
    DA(c->dt, ns_ * sizeof(double));
    DA(c->cmax, ns_ * sizeof(double));
    DA(c->last_v, ns_ * sizeof(double));
    DA(c->last_a, ns_ * sizeof(double));
    DA(c->vmax, ns_ * sizeof(unsigned long long));
    DA(c->amax, ns_ * sizeof(unsigned long long));
    DA(c->done, sizeof(unsigned int));
    DA(c->bar, 2 * sizeof(unsigned int));
    CK(cudaMemsetAsync(c->bar, 0, 2 * sizeof(unsigned int), s));
    CK(cudaMemcpyAsync(c->t, t0.data(), ns_ * sizeof(double), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(c->dt, dt0.data(), ns_ * sizeof(double), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(c->cmax, cm.data(), ns_ * sizeof(double), cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(c->last_v, 0, ns_ * sizeof(double), s));
    CK(cudaMemsetAsync(c->last_a, 0, ns_ * sizeof(double), s));
    CK(cudaMemsetAsync(c->vmax, 0, ns_ * sizeof(unsigned long long), s));
    CK(cudaMemsetAsync(c->amax, 0, ns_ * sizeof(unsigned long long), s));
    CK(cudaMemsetAsync(c->done, 0, sizeof(unsigned int), s));
    // contact tables (spatial hash of 2n or more buckets, a power of two)
    if (c->contact) {
        int ts = 1024;
        while (ts < 2 * n) ts <<= 1;
        if (ts > kHashScanBlock * kHashScanBlock * 4) return fail(c, TLSPH_ERR_ARG, "too many particles for contact");
        c->tsize = ts;
        DA(c->rest, ns_ * sizeof(double));
        DA(c->hcount, ts * sizeof(int));
        DA(c->hstart, ts * sizeof(int));
        DA(c->hbsum, (ts / kHashScanBlock + 1) * sizeof(int));
        DA(c->hbucket, n * sizeof(int));
        DA(c->hslot, n * sizeof(int));
        DA(c->hlist, n * sizeof(int));
        DA(c->hcell, n * sizeof(int4));
        DA(c->accc, dim * n * sizeof(T));
        CK(cudaMemcpyAsync(c->rest, c->resth.data(), ns_ * sizeof(double), cudaMemcpyHostToDevice, s));
        CK(cudaMemsetAsync(c->accc, 0, dim * n * sizeof(T), s));
        if (!c->kfrich.empty()) {
            DA(c->kfric, ns_ * sizeof(double));
            CK(cudaMemcpyAsync(c->kfric, c->kfrich.data(), ns_ * sizeof(double), cudaMemcpyHostToDevice, s));
        }
    }
    // first moment of the corrected kernel (reference configuration)
    DA(c->S1, n * sizeof(V4<T>));
    {
        const StepArgs<T> a = make_args<T>(c);
        if (dim == 3) k_first_moment<T, 3><<<blocks_for(n), kThreads, 0, s>>>(a, (V4<T> *)c->S1);
        else k_first_moment<T, 2><<<blocks_for(n), kThreads, 0, s>>>(a, (V4<T> *)c->S1);
        CKL();
    }
    int hf[kNumFlags];
    CK(cudaMemcpyAsync(hf, c->flags, sizeof hf, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    c->parity = 0;
    c->steps = 0;
    c->bytes_per_step = algorithmic_bytes(c, sizeof(T));
    if (hf[kFlagBounds]) return fail(c, TLSPH_ERR_STATE, "%d neighbour indices out of range in the setup", hf[kFlagBounds]);
    if (hf[kFlagCoincident])
        return fail(c, TLSPH_ERR_ARG, "%d particle pairs share a reference position", hf[kFlagCoincident] / 2);
    if (hf[kFlagSingular]) return fail(c, TLSPH_ERR_SINGULAR_L, "%d particles have a singular correction matrix",
                                       hf[kFlagSingular]);
    c->built = true;
    return TLSPH_OK;
}

int timing_event(tlsph_ctx *c) {
    if (c->ev_next + 2 > c->ev_pool.size()) {
        for (int q = 0; q < 256; q++) {
            cudaEvent_t e;
            cudaEventCreate(&e);
            c->ev_pool.push_back(e);
        }
    }
    int k = (int)c->ev_next;
    c->ev_next += 2;
    return k;
}

void collect_timing(tlsph_ctx *c) {
    for (auto &pr : c->ev_pending) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, c->ev_pool[pr.second], c->ev_pool[pr.second + 1]) == cudaSuccess) {
            c->ms[pr.first] += ms;
            c->cnt[pr.first]++;
        }
    }
    c->ev_pending.clear();
    c->ev_next = 0;
}

SurrogateDev sur_dev(const tlsph_ctx *c) {
    SurrogateDev d{};
    d.W = c->sur_W;
    d.bias = c->sur_bias;
    d.in_mean = c->sur_norm;
    d.in_std = c->sur_norm + 16;
    d.out_mean = c->sur_norm + 32;
    d.out_std = c->sur_norm + 48;
    d.env_lo = c->sur_norm + 64;
    d.env_hi = c->sur_norm + 80;
    d.enabled = c->sur_on ? 1 : 0;
    d.scope = c->sur_scope;
    return d;
}

template <int DIM, bool FRAC> tlsph_status launch_stress_sur(tlsph_ctx *c, const StepArgs<float> &a) {
    const bool tc = c->sur_tensor == TLSPH_TENSOR_TCGEN05;
    auto kern = tc ? k_stress_sur_tc<DIM, FRAC> : k_stress_sur<DIM, FRAC>;
    const size_t smem = tc ? sizeof(MlpTcSmem) : sizeof(MlpSmem);
    // per launch: the attribute belongs to the current device, and setting it costs no device work
    CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int threads = tc ? 128 * kTcGroups : 128;
    int nsm = 0, per_sm = 0;
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->p.device));
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
    const int64_t ctas = (c->n + threads - 1) / threads;
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((int64_t)std::max(per_sm, 1) * nsm, ctas));
    CK(cudaMemsetAsync(c->sur_nexact, 0, sizeof(unsigned), c->stream));
    kern<<<grid, threads, smem, c->stream>>>(a, sur_dev(c), c->sur_exact, c->sur_nexact, c->sur_count);
    CKL();
    // a grid-stride walk of the list, at most eight blocks per SM
    const unsigned gx = (unsigned)std::min<int64_t>(blocks_for(c->n), (int64_t)8 * std::max(nsm, 1));
    k_stress_exact<DIM, FRAC, kThreads><<<gx, kThreads, 0, c->stream>>>(a, c->sur_exact, c->sur_nexact);
    CKL();
    return TLSPH_OK;
}

// ---- contact accelerations between bodies: hash the current positions, list, sort, sum the pair forces
template <typename T, int DIM> tlsph_status contact_launches(tlsph_ctx *c, const StepArgs<T> &a) {
    const int n = (int)c->n, ts = c->tsize;
    const double dc = ex_dx(c);
    cudaStream_t s = c->stream;
    CK(cudaMemsetAsync(c->hcount, 0, ts * sizeof(int), s));
    k_contact_count<T><<<blocks_for(n, 128), 128, 0, s>>>(a, c->X0d, DIM, dc, ts, c->hcount, c->hbucket, c->hslot,
                                                          c->hcell);
    CKL();
    const int nb = (ts + kHashScanBlock - 1) / kHashScanBlock;
    k_hscan_blocks<<<nb, kHashScanBlock, 0, s>>>(ts, c->hcount, c->hstart, c->hbsum);
    CKL();
    k_hscan_sums<<<1, kHashScanBlock, 0, s>>>(nb, c->hbsum);
    CKL();
    k_hscan_add<<<nb, kHashScanBlock, 0, s>>>(ts, c->hstart, c->hbsum);
    CKL();
    k_contact_fill<<<blocks_for(n, 128), 128, 0, s>>>(n, c->hbucket, c->hslot, c->hstart, c->hlist);
    CKL();
    k_contact_sort<<<blocks_for(ts, 128), 128, 0, s>>>(ts, c->hcount, c->hstart, c->hlist);
    CKL();
    k_contact<T, DIM><<<blocks_for(n, 128), 128, 0, s>>>(a, c->X0d, dc, c->kc, c->rest, c->kfric, ts, c->hcount,
                                                         c->hstart, c->hlist, c->hcell, (T *)c->accc);
    CKL();
    return TLSPH_OK;
}

// ---- the lattice kernels (3D FP32 lattices): P rows per thread, 128 threads per block
constexpr int kLatThreads = 128;
inline unsigned lat_blocks(const tlsph_ctx *c, int P) {
    if (c->lat_cw > 0) {  // bands of (threads / cw) P lines, each cut into patches cw wide along x
        const int64_t lines = (c->n + c->lat_nx - 1) / c->lat_nx;
        const int64_t band = (int64_t)(kLatThreads / c->lat_cw) * P;
        return (unsigned)((lines + band - 1) / band * ((c->lat_nx + c->lat_cw - 1) / c->lat_cw));
    }
    const int64_t rows = (int64_t)P * c->lat_nx;
    return blocks_for((c->n + rows - 1) / rows * c->lat_nx, kLatThreads);
}
template <bool FRAC, bool VISC> tlsph_status launch_gradient_lat(tlsph_ctx *c, const StepArgs<float> &a, bool fuse) {
    const unsigned nb = lat_blocks(c, c->lat_rows_grad);
    if (c->lat_rows_grad == 2) {
        if (fuse) k_gradient_lat<float, FRAC, VISC, true, 2, kLatThreads><<<nb, kLatThreads, 0, c->stream>>>(a);
        else k_gradient_lat<float, FRAC, VISC, false, 2, kLatThreads><<<nb, kLatThreads, 0, c->stream>>>(a);
    } else {
        if (fuse) k_gradient_lat<float, FRAC, VISC, true, 1, kLatThreads><<<nb, kLatThreads, 0, c->stream>>>(a);
        else k_gradient_lat<float, FRAC, VISC, false, 1, kLatThreads><<<nb, kLatThreads, 0, c->stream>>>(a);
    }
    CKL();
    return TLSPH_OK;
}
template <bool FRAC> tlsph_status launch_pass2_lat(tlsph_ctx *c, const StepArgs<float> &a) {
    if (c->lat_zc > 0) {  // a column of zc planes per thread
        const int64_t nz = (c->n + c->lat_nxny - 1) / c->lat_nxny;
        const unsigned nb = blocks_for((int64_t)c->lat_nxny * ((nz + c->lat_zc - 1) / c->lat_zc), kLatThreads);
        if (c->has_visc) k_pass2_zs<float, FRAC, true, kLatThreads><<<nb, kLatThreads, 0, c->stream>>>(a);
        else k_pass2_zs<float, FRAC, false, kLatThreads><<<nb, kLatThreads, 0, c->stream>>>(a);
        CKL();
        return TLSPH_OK;
    }
    const unsigned nb = lat_blocks(c, c->lat_rows_force);
    if (c->lat_rows_force == 4) {
        if (c->has_visc) k_pass2_lat<float, FRAC, true, 4, kLatThreads><<<nb, kLatThreads, 0, c->stream>>>(a);
        else k_pass2_lat<float, FRAC, false, 4, kLatThreads><<<nb, kLatThreads, 0, c->stream>>>(a);
    } else if (c->lat_rows_force == 2) {
        if (c->has_visc) k_pass2_lat<float, FRAC, true, 2, kLatThreads><<<nb, kLatThreads, 0, c->stream>>>(a);
        else k_pass2_lat<float, FRAC, false, 2, kLatThreads><<<nb, kLatThreads, 0, c->stream>>>(a);
    } else {
        if (c->has_visc) k_pass2_lat<float, FRAC, true, 1, kLatThreads><<<nb, kLatThreads, 0, c->stream>>>(a);
        else k_pass2_lat<float, FRAC, false, 1, kLatThreads><<<nb, kLatThreads, 0, c->stream>>>(a);
    }
    CKL();
    return TLSPH_OK;
}

// ---- one step as three kernel launches (gradient, stress, force-and-damage); on a 3D FP32 lattice two
// (the stress in the tail of the gradient kernel) unless the surrogate serves the stress
template <typename T, int DIM, bool FRAC, int BS>
tlsph_status step_launches(tlsph_ctx *c, int64_t nsteps, bool timing) {
    const unsigned nb = blocks_for(c->n, BS);
    for (int64_t k = 0; k < nsteps; k++) {
        StepArgs<T> a = make_step_args<T>(c);
        int ev[3] = {-1, -1, -1};
        if (timing && c->ev_next + 6 > 4096) {
            cudaStreamSynchronize(c->stream);
            collect_timing(c);
        }
        // timing category: 0 force-and-damage pass, 1 deformation gradient, 2 stress
        auto start = [&](int cat) {
            if (!timing) return;
            ev[cat] = timing_event(c);
            cudaEventRecord(c->ev_pool[ev[cat]], c->stream);
        };
        auto stop = [&](int cat) {
            if (!timing) return;
            cudaEventRecord(c->ev_pool[ev[cat] + 1], c->stream);
            c->ev_pending.push_back({cat, ev[cat]});
        };
        start(1);
        if (c->nexlist > 0) {  // boundary values given by expressions, from the state at the step's start
            k_expr_bcs<T, DIM><<<blocks_for(c->nexlist, 128), 128, 0, c->stream>>>(
                a, c->exlist, c->nexlist, c->X0d, c->excode, c->exK, c->exprog, ex_dx(c), c->exval, c->exskip);
            CKL();
        }
        if (c->leap) {  // Algorithm 2, predictor (timed with the deformation gradient)
            k_predict<T, DIM, FRAC, BS><<<nb, BS, 0, c->stream>>>(a);
            CKL();
        }
        if (c->contact) {  // contact between bodies at the level of the forces
            tlsph_status st = contact_launches<T, DIM>(c, a);
            if (st != TLSPH_OK) return st;
        }
        constexpr bool lat_ok = DIM == 3 && std::is_same<T, float>::value;
        const bool lat = lat_ok && a.lat_nx > 0;
        const bool fused = lat && c->fuse_stress && !c->sur_on;
        if constexpr (lat_ok) {
            if (lat) {
                tlsph_status st = c->has_visc ? launch_gradient_lat<FRAC, true>(c, a, fused)
                                              : launch_gradient_lat<FRAC, false>(c, a, fused);
                if (st != TLSPH_OK) return st;
            }
        }
        if (!lat) {
            if (c->has_visc) k_gradient<T, DIM, FRAC, true, BS><<<nb, BS, 0, c->stream>>>(a);
            else k_gradient<T, DIM, FRAC, false, BS><<<nb, BS, 0, c->stream>>>(a);
            CKL();
        }
        stop(1);
        if (!fused) {
            start(2);
            bool done_sur = false;
            if constexpr (std::is_same<T, float>::value) {
                if (c->sur_on) {
                    tlsph_status st = launch_stress_sur<DIM, FRAC>(c, a);
                    if (st != TLSPH_OK) return st;
                    done_sur = true;
                }
            }
            if (!done_sur) {
                k_stress<T, DIM, FRAC, false, BS><<<nb, BS, 0, c->stream>>>(a);
                CKL();
            }
            stop(2);
        }
        start(0);
        if constexpr (lat_ok) {
            if (lat) {
                tlsph_status st = launch_pass2_lat<FRAC>(c, a);
                if (st != TLSPH_OK) return st;
            }
        }
        if (!lat) {
            if (c->has_visc) k_pass2<T, DIM, FRAC, true, BS><<<nb, BS, 0, c->stream>>>(a);
            else k_pass2<T, DIM, FRAC, false, BS><<<nb, BS, 0, c->stream>>>(a);
            CKL();
        }
        stop(0);
        if (!c->leap) c->parity ^= 1;
        c->steps++;
    }
    return TLSPH_OK;
}

// ---- steps replayed from a CUDA graph holding two steps (the ping-pong returns to parity 0)
template <typename T, int DIM, bool FRAC, int BS>
tlsph_status step_graph(tlsph_ctx *c, int64_t nsteps) {
    if (nsteps > 0 && c->parity == 1) {
        tlsph_status st = step_launches<T, DIM, FRAC, BS>(c, 1, false);
        if (st != TLSPH_OK) return st;
        nsteps--;
    }
    if (nsteps >= 2 && !c->gexec) {
        cudaGraph_t g = nullptr;
        const int par = c->parity;
        const int64_t steps = c->steps, launches = c->launches;
        CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
        tlsph_status st = step_launches<T, DIM, FRAC, BS>(c, 2, false);
        cudaError_t e = cudaStreamEndCapture(c->stream, &g);
        c->graph_launches = c->launches - launches;
        c->parity = par;
        c->steps = steps;
        c->launches = launches;
        if (st != TLSPH_OK) return st;
        if (e != cudaSuccess) return fail(c, TLSPH_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
        e = cudaGraphInstantiate(&c->gexec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            c->gexec = nullptr;
            return fail(c, TLSPH_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
        }
    }
    for (; nsteps >= 2; nsteps -= 2) {
        CK(cudaGraphLaunch(c->gexec, c->stream));
        c->launches += c->graph_launches;
        c->steps += 2;
    }
    if (nsteps) return step_launches<T, DIM, FRAC, BS>(c, nsteps, false);
    return TLSPH_OK;
}

// ---- steps in one cooperative persistent launch (all blocks resident, bounded grid barriers)
template <typename T, int DIM, bool FRAC, bool VISC, int BS>
tlsph_status step_persistent_v(tlsph_ctx *c, int64_t nsteps) {
    auto kern = k_persistent<T, DIM, FRAC, VISC, BS>;
    int per_sm = 0, nsm = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, BS, 0));
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->p.device));
    const int64_t tiles = (c->n + BS - 1) / BS;
    const int grid = (int)std::min<int64_t>((int64_t)per_sm * nsm, tiles);
    if (grid < 1) return fail(c, TLSPH_ERR_CUDA, "persistent kernel cannot be resident");
    GridBarrier bar{c->bar, c->bar + 1, (unsigned)grid + (c->barrier_test ? 1u : 0u), 2000000000LL};
    while (nsteps > 0) {
        const int chunk = (int)std::min<int64_t>(nsteps, 1 << 20);
        StepArgs<T> a = make_args<T>(c);
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)grid);
        cfg.blockDim = dim3(BS);
        cfg.stream = c->stream;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        CK(cudaLaunchKernelEx(&cfg, kern, a, chunk, bar));
        CKL();
        if (chunk & 1) c->parity ^= 1;
        c->steps += chunk;
        nsteps -= chunk;
    }
    return TLSPH_OK;
}

template <typename T, int DIM, bool FRAC, int BS>
tlsph_status step_mode(tlsph_ctx *c, int64_t nsteps) {
    if (c->mode == TLSPH_MODE_GRAPH && !c->timing) return step_graph<T, DIM, FRAC, BS>(c, nsteps);
    if (c->mode == TLSPH_MODE_PERSISTENT) {
        if (BS == 64) return fail(c, TLSPH_ERR_ARG, "the persistent mode needs a block of 128 or 256");
        if (c->leap) return fail(c, TLSPH_ERR_ARG, "the persistent mode runs Algorithm 1 only");
        if (c->nexlist > 0)
            return fail(c, TLSPH_ERR_ARG, "the persistent mode takes no boundary conditions given by expressions");
        if (c->contact) return fail(c, TLSPH_ERR_ARG, "the persistent mode takes no contact between bodies");
        return c->has_visc ? step_persistent_v<T, DIM, FRAC, true, (BS < 128 ? 128 : BS)>(c, nsteps)
                           : step_persistent_v<T, DIM, FRAC, false, (BS < 128 ? 128 : BS)>(c, nsteps);
    }
    return step_launches<T, DIM, FRAC, BS>(c, nsteps, c->timing);
}

template <typename T, int DIM, bool FRAC> tlsph_status step_dim(tlsph_ctx *c, int64_t nsteps) {
    switch (c->bs) {
    case 64: return step_mode<T, DIM, FRAC, 64>(c, nsteps);
    case 256: return step_mode<T, DIM, FRAC, 256>(c, nsteps);
    default: return step_mode<T, DIM, FRAC, 128>(c, nsteps);
    }
}

template <typename T> tlsph_status step_impl(tlsph_ctx *c, int64_t nsteps) {
    if (c->p.dim == 3) return c->has_frac ? step_dim<T, 3, true>(c, nsteps) : step_dim<T, 3, false>(c, nsteps);
    return c->has_frac ? step_dim<T, 2, true>(c, nsteps) : step_dim<T, 2, false>(c, nsteps);
}

template <typename T> tlsph_status diag_pass(tlsph_ctx *c) {
    const int64_t n = c->n;
    if (!c->Fd) {
        DA(c->Fd, 9 * n * sizeof(T));
        DA(c->Pd, 9 * n * sizeof(T));
        DA(c->psid, n * sizeof(T));
    }
    StepArgs<T> a = make_args<T>(c);
    const unsigned nb = blocks_for(n);
    if (c->p.dim == 3) {
        k_gradient<T, 3, false, false, kThreads><<<nb, kThreads, 0, c->stream>>>(a);
        CKL();
        if (c->has_frac) k_stress<T, 3, true, true, kThreads><<<nb, kThreads, 0, c->stream>>>(a);
        else k_stress<T, 3, false, true, kThreads><<<nb, kThreads, 0, c->stream>>>(a);
    } else {
        k_gradient<T, 2, false, false, kThreads><<<nb, kThreads, 0, c->stream>>>(a);
        CKL();
        if (c->has_frac) k_stress<T, 2, true, true, kThreads><<<nb, kThreads, 0, c->stream>>>(a);
        else k_stress<T, 2, false, true, kThreads><<<nb, kThreads, 0, c->stream>>>(a);
    }
    CKL();
    return TLSPH_OK;
}

template <typename T> tlsph_status energies_impl(tlsph_ctx *c, double *out) {
    tlsph_status st = diag_pass<T>(c);
    if (st != TLSPH_OK) return st;
    CK(cudaMemsetAsync(c->energy, 0, 8 * sizeof(double), c->stream));
    StepArgs<T> a = make_args<T>(c);
    const unsigned nb = blocks_for(c->n);
    if (c->p.dim == 3) {
        if (c->has_frac) k_energy<T, 3, true><<<nb, kThreads, 0, c->stream>>>(a, c->energy);
        else k_energy<T, 3, false><<<nb, kThreads, 0, c->stream>>>(a, c->energy);
    } else {
        if (c->has_frac) k_energy<T, 2, true><<<nb, kThreads, 0, c->stream>>>(a, c->energy);
        else k_energy<T, 2, false><<<nb, kThreads, 0, c->stream>>>(a, c->energy);
    }
    CKL();
    double e[5];
    CK(cudaMemcpyAsync(e, c->energy, sizeof e, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(&out[5], c->t, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    for (int q = 0; q < 5; q++) out[q] = e[q];
    return TLSPH_OK;
}

int field_comps(const tlsph_ctx *c, int field) {
    switch (field) {
    case TLSPH_FIELD_U:
    case TLSPH_FIELD_V:
    case TLSPH_FIELD_X:
    case TLSPH_FIELD_ACC: return c->p.dim;
    case TLSPH_FIELD_S:
    case TLSPH_FIELD_SDOT:
    case TLSPH_FIELD_H:
    case TLSPH_FIELD_EPSP: return 1;
    case TLSPH_FIELD_P:
    case TLSPH_FIELD_F:
    case TLSPH_FIELD_CPINV: return 9;
    default: return -1;
    }
}

size_t state_bytes(const tlsph_ctx *c) {
    const size_t ts = c->p.precision == TLSPH_FP64 ? 8 : 4, n = (size_t)c->n;
    return 64 + n * (3 * 8 + 2 * 4 * ts + ts * (1 + 1 + 6 + 1) + 8) + (size_t)c->nspec * 2 * 8 +
           (c->leap ? (size_t)c->p.dim * n * ts : 0);
}

template <typename T> tlsph_status read_impl(tlsph_ctx *c, int field, double *dst /* device, caller order */) {
    const int64_t n = c->n;
    const int dim = c->p.dim;
    const unsigned nb = blocks_for(n);
    cudaStream_t s = c->stream;
    switch (field) {
    case TLSPH_FIELD_U: k_to_caller<double><<<nb, kThreads, 0, s>>>(n, dim, c->u64, n, c->perm, dst); break;
    case TLSPH_FIELD_X: k_x_to_caller<<<nb, kThreads, 0, s>>>(n, dim, c->X0d, c->u64, c->perm, dst); break;
    case TLSPH_FIELD_V:
        k_v4_to_caller<T><<<nb, kThreads, 0, s>>>(n, dim, 0, (const V4<T> *)c->vs[c->parity], c->perm, dst);
        break;
    case TLSPH_FIELD_S:
        k_v4_to_caller<T><<<nb, kThreads, 0, s>>>(n, 1, 3, (const V4<T> *)c->vs[c->parity], c->perm, dst);
        break;
    case TLSPH_FIELD_SDOT: k_to_caller<T><<<nb, kThreads, 0, s>>>(n, 1, (const T *)c->sdot, n, c->perm, dst); break;
    case TLSPH_FIELD_H: k_to_caller<T><<<nb, kThreads, 0, s>>>(n, 1, (const T *)c->H, n, c->perm, dst); break;
    case TLSPH_FIELD_EPSP: k_to_caller<T><<<nb, kThreads, 0, s>>>(n, 1, (const T *)c->ep, n, c->perm, dst); break;
    case TLSPH_FIELD_ACC: k_to_caller<T><<<nb, kThreads, 0, s>>>(n, dim, (const T *)c->accd, n, c->perm, dst); break;
    case TLSPH_FIELD_CPINV: k_cpinv_to_caller<T><<<nb, kThreads, 0, s>>>(n, (const T *)c->K, c->perm, dst); break;
    case TLSPH_FIELD_F:
    case TLSPH_FIELD_P: {
        tlsph_status st = diag_pass<T>(c);
        if (st != TLSPH_OK) return st;
        k_to_caller<T><<<nb, kThreads, 0, s>>>(n, 9, (const T *)(field == TLSPH_FIELD_F ? c->Fd : c->Pd), n, c->perm,
                                                dst);
        break;
    }
    default: return fail(c, TLSPH_ERR_ARG, "field %d cannot be read", field);
    }
    CKL();
    return TLSPH_OK;
}

template <typename T> tlsph_status write_impl(tlsph_ctx *c, int field, const double *src /* device */) {
    const int64_t n = c->n;
    const int dim = c->p.dim;
    const unsigned nb = blocks_for(n);
    cudaStream_t s = c->stream;
    switch (field) {
    case TLSPH_FIELD_U:
        k_from_caller<double><<<nb, kThreads, 0, s>>>(n, dim, src, c->perm, c->u64, n);
        CKL();
        k_refresh_ug<T><<<nb, kThreads, 0, s>>>(n, dim, c->u64, (V4<T> *)c->ug[c->parity]);
        break;
    case TLSPH_FIELD_V: k_v4_from_caller<T><<<nb, kThreads, 0, s>>>(n, dim, 0, src, c->perm, (V4<T> *)c->vs[c->parity]); break;
    case TLSPH_FIELD_S: k_v4_from_caller<T><<<nb, kThreads, 0, s>>>(n, 1, 3, src, c->perm, (V4<T> *)c->vs[c->parity]); break;
    case TLSPH_FIELD_SDOT: k_from_caller<T><<<nb, kThreads, 0, s>>>(n, 1, src, c->perm, (T *)c->sdot, n); break;
    case TLSPH_FIELD_H: k_from_caller<T><<<nb, kThreads, 0, s>>>(n, 1, src, c->perm, (T *)c->H, n); break;
    case TLSPH_FIELD_EPSP: k_from_caller<T><<<nb, kThreads, 0, s>>>(n, 1, src, c->perm, (T *)c->ep, n); break;
    case TLSPH_FIELD_CPINV: k_cpinv_from_caller<T><<<nb, kThreads, 0, s>>>(n, src, c->perm, (T *)c->K); break;
    default: return fail(c, TLSPH_ERR_ARG, "field %d cannot be written", field);
    }
    CKL();
    return TLSPH_OK;
}

// checkpoint blob: header, u64, ug, vs, sdot, H, K, ep, t, dt (sorted order)
template <typename T> tlsph_status state_io(tlsph_ctx *c, char *blob /* host */, bool save) {
    const size_t n = (size_t)c->n, ts = sizeof(T);
    struct Part { void *p; size_t bytes; };
    Part parts[] = {{c->u64, 3 * n * 8},          {c->ug[c->parity], n * sizeof(V4<T>)},
                    {c->vs[c->parity], n * sizeof(V4<T>)}, {c->sdot, n * ts},
                    {c->H, n * ts},               {c->K, 6 * n * ts},
                    {c->ep, n * ts},              {c->t, (size_t)c->nspec * 8},
                    {c->dt, (size_t)c->nspec * 8},
                    {c->accd, c->leap ? (size_t)c->p.dim * n * ts : 0},  // a_{n-1/2} of Algorithm 2
                    {c->wext, n * 8}};
    int64_t hdr[8] = {0x54534c50485354LL, (int64_t)n, c->p.precision, c->nspec, c->steps, c->p.dim, 0, 0};
    cudaStream_t s = c->stream;
    if (save) {
        memcpy(blob, hdr, sizeof hdr);
    } else {
        int64_t h2[8];
        memcpy(h2, blob, sizeof h2);
        if (h2[0] != hdr[0] || h2[1] != hdr[1] || h2[2] != hdr[2] || h2[3] != hdr[3] || h2[5] != hdr[5])
            return fail(c, TLSPH_ERR_ARG, "checkpoint does not match this context");
        c->steps = h2[4];
    }
    size_t off = 64;
    for (const Part &pt : parts) {
        if (save) CK(cudaMemcpyAsync(blob + off, pt.p, pt.bytes, cudaMemcpyDeviceToHost, s));
        else CK(cudaMemcpyAsync(pt.p, blob + off, pt.bytes, cudaMemcpyHostToDevice, s));
        off += pt.bytes;
    }
    CK(cudaStreamSynchronize(s));
    return TLSPH_OK;
}

tlsph_status check_flags(tlsph_ctx *c) {
    int hf[kNumFlags];
    CK(cudaMemcpyAsync(hf, c->flags, sizeof hf, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    int64_t dn = hf[kFlagNonfinite] - c->flags_seen[kFlagNonfinite];
    int64_t dc = hf[kFlagNoconv] - c->flags_seen[kFlagNoconv];
    int64_t dt = hf[kFlagTimeout] - c->flags_seen[kFlagTimeout];
    int64_t db = hf[kFlagBounds] - c->flags_seen[kFlagBounds];
    for (int q = 0; q < kNumFlags; q++) c->flags_seen[q] = hf[q];
    if (db > 0) return fail(c, TLSPH_ERR_STATE, "%lld neighbour indices out of range (debug build)", (long long)db);
    if (dt > 0) {
        // a persistent launch gave up at a barrier: its steps are incomplete; reset the
        // barrier and the timeout flag so that the context stays usable
        CK(cudaMemsetAsync(c->bar, 0, 2 * sizeof(unsigned int), c->stream));
        CK(cudaMemsetAsync(c->flags + kFlagTimeout, 0, sizeof(int), c->stream));
        CK(cudaStreamSynchronize(c->stream));
        c->flags_seen[kFlagTimeout] = 0;
        return fail(c, TLSPH_ERR_TIMEOUT, "a grid barrier of the persistent step gave up after its time limit");
    }
    if (dn > 0) return fail(c, TLSPH_ERR_NONFINITE, "%lld non-finite stresses or accelerations", (long long)dn);
    if (dc > 0) return fail(c, TLSPH_ERR_NOCONVERGE, "%lld J2 return maps did not converge", (long long)dc);
    return TLSPH_OK;
}

// Autotuner: time every execution mode / block size on the live problem for a few steps,
// each from the same snapshot of the evolving state, keep the fastest, restore the state.
struct Snap {
    void *p;
    size_t bytes;
};
template <typename T> std::vector<Snap> snap_parts(tlsph_ctx *c) {
    const size_t n = (size_t)c->n, ns = (size_t)c->nspec, ts = sizeof(T);
    return {{c->u64, 3 * n * 8},       {c->ug[c->parity], n * sizeof(V4<T>)}, {c->vs[c->parity], n * sizeof(V4<T>)},
            {c->accd, c->leap ? (size_t)c->p.dim * n * ts : 0},
            {c->sdot, n * ts},         {c->H, n * ts},                         {c->K, 6 * n * ts},
            {c->ep, n * ts},           {c->t, ns * 8},                         {c->dt, ns * 8},
            {c->vmax, ns * 8},         {c->amax, ns * 8},                      {c->last_v, ns * 8},
            {c->last_a, ns * 8},       {c->flags, kNumFlags * sizeof(int)},     {c->done, sizeof(unsigned int)},
            {c->bar, 2 * sizeof(unsigned int)}, {c->wext, n * 8}};
}

template <typename T>
tlsph_status autotune_impl(tlsph_ctx *c, int trial, tlsph_tuning *best, tlsph_tuning *all) {
    std::vector<Snap> parts = snap_parts<T>(c);
    size_t total = 0;
    for (const Snap &q : parts) total += (q.bytes + 255) / 256 * 256;
    char *snap = nullptr;
    if (cudaMalloc(&snap, total) != cudaSuccess) {
        cudaGetLastError();
        return fail(c, TLSPH_ERR_OOM, "autotune snapshot");
    }
    const int par = c->parity, mode0 = c->mode, bs0 = c->bs;
    const int64_t steps = c->steps;
    int64_t seen[kNumFlags];
    for (int q = 0; q < kNumFlags; q++) seen[q] = c->flags_seen[q];
    auto copy_all = [&](bool save) {
        size_t off = 0;
        for (const Snap &q : parts) {
            if (save) cudaMemcpyAsync(snap + off, q.p, q.bytes, cudaMemcpyDeviceToDevice, c->stream);
            else cudaMemcpyAsync(q.p, snap + off, q.bytes, cudaMemcpyDeviceToDevice, c->stream);
            off += (q.bytes + 255) / 256 * 256;
        }
    };
    auto restore = [&]() {
        c->parity = par;  // the snapshot holds the buffers of this parity
        copy_all(false);
        c->steps = steps;
        for (int q = 0; q < kNumFlags; q++) c->flags_seen[q] = seen[q];
        drop_graph(c);
    };
    copy_all(true);
    const int cand[6][2] = {{TLSPH_MODE_LAUNCH, 64},  {TLSPH_MODE_LAUNCH, 128},     {TLSPH_MODE_LAUNCH, 256},
                            {TLSPH_MODE_GRAPH, 128},  {TLSPH_MODE_PERSISTENT, 128}, {TLSPH_MODE_PERSISTENT, 256}};
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double best_ms = INFINITY;
    int bi = -1;
    const bool timing = c->timing;
    c->timing = false;
    for (int k = 0; k < 6; k++) {
        c->mode = cand[k][0];
        c->bs = cand[k][1];
        drop_graph(c);
        double ms_step = INFINITY;
        tlsph_status st = step_impl<T>(c, 2);
        if (st == TLSPH_OK) {
            cudaEventRecord(e0, c->stream);
            st = step_impl<T>(c, trial);
            cudaEventRecord(e1, c->stream);
        }
        if (st == TLSPH_OK && cudaStreamSynchronize(c->stream) == cudaSuccess && check_flags(c) == TLSPH_OK) {
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            ms_step = ms / trial;
        }
        cudaGetLastError();
        if (all) all[k] = tlsph_tuning{cand[k][0], cand[k][1], ms_step};
        if (ms_step < best_ms) {
            best_ms = ms_step;
            bi = k;
        }
        restore();
    }
    c->timing = timing;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamSynchronize(c->stream);
    cudaFree(snap);
    if (bi < 0) {
        c->mode = mode0;
        c->bs = bs0;
        return fail(c, TLSPH_ERR_CUDA, "no execution mode ran");
    }
    c->mode = cand[bi][0];
    c->bs = cand[bi][1];
    if (best) *best = tlsph_tuning{c->mode, c->bs, best_ms};
    return TLSPH_OK;
}

template <typename T> tlsph_status apply_expr_impl(tlsph_ctx *c, int field, const int ids[3]) {
    tlsph_status st = ex_sync(c);
    if (st != TLSPH_OK) return st;
    StepArgs<T> a = make_args<T>(c);
    const int3 id3 = make_int3(ids[0], ids[1], ids[2]);
    const int f = field == TLSPH_FIELD_U ? 0 : 1;
    V4<T> *ug = (V4<T> *)c->ug[c->parity], *vs = (V4<T> *)c->vs[c->parity];
    const unsigned nb = blocks_for(c->n, 128);
    if (c->p.dim == 3)
        k_expr_field<T, 3><<<nb, 128, 0, c->stream>>>(a, c->X0d, c->excode, c->exK, c->exprog, id3, ex_dx(c), f, ug, vs);
    else
        k_expr_field<T, 2><<<nb, 128, 0, c->stream>>>(a, c->X0d, c->excode, c->exK, c->exprog, id3, ex_dx(c), f, ug, vs);
    CKL();
    CK(cudaStreamSynchronize(c->stream));
    return TLSPH_OK;
}

}  // namespace

// ===================================================================== C-ABI
extern "C" {

tlsph_status tlsph_create(const tlsph_params *params, tlsph_ctx **out) {
    if (!out) return TLSPH_ERR_ARG;
    *out = nullptr;
    if (!params || (params->dim != 2 && params->dim != 3) || !(params->h > 0.0) || !(params->support > 0.0) ||
        (params->precision != TLSPH_FP64 && params->precision != TLSPH_FP32_U64) ||
        params->integrator < 0 || params->integrator > 2 || params->dt_mode < 0 || params->dt_mode > 2 ||
        (params->dt_mode == TLSPH_DT_FIXED && !(params->fixed_dt > 0.0)) ||
        (params->dt_mode != TLSPH_DT_FIXED && !(params->cfl > 0.0)))
        return TLSPH_ERR_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || params->device < 0 || params->device >= ndev) {
        cudaGetLastError();
        return TLSPH_ERR_CUDA;
    }
    if (cudaSetDevice(params->device) != cudaSuccess) return TLSPH_ERR_CUDA;
    tlsph_ctx *c = new tlsph_ctx();
    c->p = *params;
    c->leap = params->integrator == TLSPH_INTEGRATOR_LEAPFROG;
    if (params->cuda_stream) {
        c->stream = (cudaStream_t)params->cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete c;
            return TLSPH_ERR_CUDA;
        }
        c->own_stream = true;
    }
    *out = c;
    return TLSPH_OK;
}

void tlsph_destroy(tlsph_ctx *c) {
    if (!c) return;
    cudaSetDevice(c->p.device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    free_device(c);
    free_ex_tables(c);
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
}

const char *tlsph_last_error(const tlsph_ctx *c) { return c ? c->err.c_str() : "null context"; }

tlsph_status tlsph_set_materials(tlsph_ctx *c, int n, const tlsph_material *m) {
    if (!c) return TLSPH_ERR_ARG;
    if (n <= 0 || n > 65535 || !m) return fail(c, TLSPH_ERR_ARG, "bad material table");
    for (int i = 0; i < n; i++) {
        if (!(m[i].E > 0.0) || !(m[i].nu > -1.0 && m[i].nu < 0.5) || !(m[i].rho > 0.0))
            return fail(c, TLSPH_ERR_ARG, "material %d: need E > 0, -1 < nu < 0.5, rho > 0", i);
        if (m[i].model != TLSPH_MODEL_SVK && m[i].model != TLSPH_MODEL_NH && m[i].model != TLSPH_MODEL_J2)
            return fail(c, TLSPH_ERR_ARG, "material %d: unknown model %d", i, m[i].model);
        if (m[i].model == TLSPH_MODEL_J2 && !(m[i].sigma_y0 > 0.0))
            return fail(c, TLSPH_ERR_ARG, "material %d: J2 needs sigma_y0 > 0", i);
        if (m[i].fracture && m[i].model != TLSPH_MODEL_J2 && (!(m[i].Gc > 0.0) || !(m[i].eps0 > 0.0)))
            return fail(c, TLSPH_ERR_ARG, "material %d: fracture needs Gc > 0 and eps0 > 0", i);
    }
    c->mats.assign(m, m + n);
    c->built = false;
    return TLSPH_OK;
}

tlsph_status tlsph_create_particles(tlsph_ctx *c, int64_t n, const double *X0, const double *vol, const double *v0,
                                    const int32_t *material_id, const int32_t *specimen_id) {
    if (!c) return TLSPH_ERR_ARG;
    if (c->mats.empty()) return fail(c, TLSPH_ERR_STATE, "set_materials must come before create_particles");
    if (n <= 0 || n >= (int64_t)1 << 31 || !X0 || !vol || !material_id)
        return fail(c, TLSPH_ERR_ARG, "create_particles: bad size or null array");
    const int d = c->p.dim;
    c->n = n;
    c->X0h.assign(3 * n, 0.0);
    c->volh.assign(vol, vol + n);
    c->midh.assign(material_id, material_id + n);
    c->spech.assign(n, 0);
    c->v0h.clear();
    if (v0) c->v0h.assign(v0, v0 + n * d);
    c->nspec = 1;
    for (int64_t i = 0; i < n; i++) {
        for (int k = 0; k < d; k++) {
            double x = X0[d * i + k];
            if (!std::isfinite(x)) return fail(c, TLSPH_ERR_ARG, "particle %lld: non-finite position", (long long)i);
            c->X0h[3 * i + k] = x;
        }
        if (!(vol[i] > 0.0)) return fail(c, TLSPH_ERR_ARG, "particle %lld: volume must be > 0", (long long)i);
        if (material_id[i] < 0 || material_id[i] >= (int)c->mats.size())
            return fail(c, TLSPH_ERR_ARG, "particle %lld: material id out of range", (long long)i);
        if (specimen_id) {
            if (specimen_id[i] < 0) return fail(c, TLSPH_ERR_ARG, "particle %lld: negative specimen id", (long long)i);
            c->spech[i] = specimen_id[i];
            c->nspec = std::max(c->nspec, specimen_id[i] + 1);
        }
    }
    c->bcs.clear();
    c->notches.clear();
    free_device(c);
    return TLSPH_OK;
}

tlsph_status tlsph_add_bc(tlsph_ctx *c, const uint8_t *mask, int kind, int comp_mask, const double value[3],
                          double t_start, double t_end, double ramp, double area) {
    if (!c) return TLSPH_ERR_ARG;
    if (c->n <= 0) return fail(c, TLSPH_ERR_STATE, "create_particles must come before add_bc");
    if (!mask || !value || kind < 0 || kind > 4) return fail(c, TLSPH_ERR_ARG, "add_bc: bad kind or null array");
    if (kind == TLSPH_BC_PHASE_BOUND && !(comp_mask & 1))
        return fail(c, TLSPH_ERR_ARG, "add_bc: a phase-field bound acts on component 0 (bit 0 of comp_mask)");
    if (kind == TLSPH_BC_PHASE_BOUND && !(value[0] >= 0.0 && value[0] <= 1.0))
        return fail(c, TLSPH_ERR_ARG, "add_bc: a phase-field bound takes a value in [0, 1]");
    if (c->bcs.size() >= 32767) return fail(c, TLSPH_ERR_ARG, "too many boundary conditions");
    BCHost b;
    b.kind = kind;
    b.comp_mask = comp_mask;
    for (int q = 0; q < 3; q++) b.value[q] = value[q];
    b.t_start = t_start;
    b.t_end = t_end;
    b.ramp = ramp;
    b.area = area;
    for (int64_t i = 0; i < c->n; i++)
        if (mask[i]) b.ids.push_back(i);
    b.count = (int64_t)b.ids.size();
    c->bcs.push_back(std::move(b));
    c->built = false;
    return TLSPH_OK;
}

tlsph_status tlsph_add_notch(tlsph_ctx *c, const double quad[12]) {
    if (!c) return TLSPH_ERR_ARG;
    if (!quad || c->notches.size() / 12 >= 512) return fail(c, TLSPH_ERR_ARG, "add_notch: null or more than 512");
    for (int k = 0; k < 12; k++)
        if (!std::isfinite(quad[k])) return fail(c, TLSPH_ERR_ARG, "add_notch: non-finite coordinate %d", k);
    c->notches.insert(c->notches.end(), quad, quad + 12);
    c->built = false;
    return TLSPH_OK;
}

tlsph_status tlsph_expr_check(const char *locals, const char *expr, char *msg, size_t msg_len) {
    if (!expr) return TLSPH_ERR_ARG;
    ExCompiler comp;
    ExProgram prog;
    std::string err;
    const bool ok = comp.compile(locals ? locals : "", expr, prog, err);
    if (msg && msg_len) snprintf(msg, msg_len, "%s", ok ? "" : err.c_str());
    return ok ? TLSPH_OK : TLSPH_ERR_ARG;
}

tlsph_status tlsph_expr_compile(tlsph_ctx *c, const char *locals, const char *expr, int *id) {
    if (!c) return TLSPH_ERR_ARG;
    if (!expr || !id) return fail(c, TLSPH_ERR_ARG, "expr_compile: null expression or id");
    if (c->exprogs.size() >= 4096) return fail(c, TLSPH_ERR_ARG, "too many expressions");
    ExCompiler comp;
    ExProgram prog;
    std::string err;
    if (!comp.compile(locals ? locals : "", expr, prog, err)) return fail(c, TLSPH_ERR_ARG, "expression: %s", err.c_str());
    c->exprogs.push_back(std::move(prog));
    c->ex_dirty = true;
    *id = (int)c->exprogs.size() - 1;
    return TLSPH_OK;
}

tlsph_status tlsph_add_bc_expr(tlsph_ctx *c, const uint8_t *mask, int kind, int comp_mask, const int expr_id[3],
                               double t_start, double t_end, double area) {
    if (!c) return TLSPH_ERR_ARG;
    if (!expr_id) return fail(c, TLSPH_ERR_ARG, "add_bc_expr: null expression ids");
    const int dim = c->p.dim;
    if (comp_mask <= 0 || comp_mask >= (1 << dim)) return fail(c, TLSPH_ERR_ARG, "add_bc_expr: bad component mask");
    for (int q = 0; q < dim; q++)
        if ((comp_mask >> q) & 1)
            if (expr_id[q] < 0 || expr_id[q] >= (int)c->exprogs.size())
                return fail(c, TLSPH_ERR_ARG, "add_bc_expr: component %d has no compiled expression", q);
    const double zero[3] = {0.0, 0.0, 0.0};
    tlsph_status st = tlsph_add_bc(c, mask, kind, comp_mask, zero, t_start, t_end, 0.0, area);
    if (st != TLSPH_OK) return st;
    for (int q = 0; q < 3; q++) c->bcs.back().expr[q] = (q < dim && ((comp_mask >> q) & 1)) ? expr_id[q] : -1;
    return TLSPH_OK;
}

tlsph_status tlsph_apply_expr(tlsph_ctx *c, int field, const int expr_id[3]) {
    DeviceScope ds_(c ? c->p.device : -1);
    if (!c) return TLSPH_ERR_ARG;
    if (!c->built) return fail(c, TLSPH_ERR_STATE, "build_ref_neighbours must come before apply_expr");
    if (!expr_id || (field != TLSPH_FIELD_U && field != TLSPH_FIELD_V))
        return fail(c, TLSPH_ERR_ARG, "apply_expr: field must be U or V");
    int ids[3] = {-1, -1, -1};
    for (int q = 0; q < c->p.dim; q++) {
        if (expr_id[q] >= (int)c->exprogs.size()) return fail(c, TLSPH_ERR_ARG, "apply_expr: unknown expression");
        ids[q] = expr_id[q] < 0 ? -1 : expr_id[q];
    }
    return c->p.precision == TLSPH_FP64 ? apply_expr_impl<double>(c, field, ids) : apply_expr_impl<float>(c, field, ids);
}

tlsph_status tlsph_expr_eval(tlsph_ctx *c, int id, int64_t n, const double *vars, double *out, uint8_t *skip) {
    DeviceScope ds_(c ? c->p.device : -1);
    if (!c) return TLSPH_ERR_ARG;
    if (id < 0 || id >= (int)c->exprogs.size()) return fail(c, TLSPH_ERR_ARG, "expr_eval: unknown expression");
    if (n < 0 || (n > 0 && (!vars || !out || !skip))) return fail(c, TLSPH_ERR_ARG, "expr_eval: bad buffers");
    if (n == 0) return TLSPH_OK;
    tlsph_status st = ex_sync(c);
    if (st != TLSPH_OK) return st;
    double *dv = nullptr, *dout = nullptr;
    uint8_t *dsk = nullptr;
    if (cudaMalloc(&dv, n * kExVars * sizeof(double)) != cudaSuccess || cudaMalloc(&dout, n * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&dsk, n) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(dv);
        cudaFree(dout);
        cudaFree(dsk);
        return fail(c, TLSPH_ERR_OOM, "expr_eval buffers");
    }
    ExProg pr{0, (int)c->exprogs[id].code.size(), 0, 0};
    for (int q = 0; q < id; q++) {
        pr.code += (int)c->exprogs[q].code.size();
        pr.consts += (int)c->exprogs[q].consts.size();
    }
    cudaMemcpyAsync(dv, vars, n * kExVars * sizeof(double), cudaMemcpyHostToDevice, c->stream);
    k_expr_rows<<<(unsigned)((n + 127) / 128), 128, 0, c->stream>>>(c->excode, c->exK, pr, n, dv, dout, dsk);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
        c->launches++;
        cudaMemcpyAsync(out, dout, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
        cudaMemcpyAsync(skip, dsk, n, cudaMemcpyDeviceToHost, c->stream);
        e = cudaStreamSynchronize(c->stream);
    }
    cudaFree(dv);
    cudaFree(dout);
    cudaFree(dsk);
    if (e != cudaSuccess) return fail(c, TLSPH_ERR_CUDA, "expr_eval: %s", cudaGetErrorString(e));
    return TLSPH_OK;
}

tlsph_status tlsph_set_contact(tlsph_ctx *c, double contcoeff, int nbodies, const double *restitution) {
    if (!c) return TLSPH_ERR_ARG;
    if (c->n <= 0) return fail(c, TLSPH_ERR_STATE, "create_particles must come before set_contact");
    if (!(contcoeff > 0.0) || nbodies != c->nspec || !restitution)
        return fail(c, TLSPH_ERR_ARG, "set_contact: need contcoeff > 0 and one restitution per specimen (%d)", c->nspec);
    if (c->p.dt_mode == TLSPH_DT_ADAPTIVE)
        return fail(c, TLSPH_ERR_ARG, "set_contact: bodies in contact share one clock; use a fixed or static step");
    for (int b = 0; b < nbodies; b++)
        if (!(restitution[b] > 0.0 && restitution[b] <= 1.0))
            return fail(c, TLSPH_ERR_ARG, "set_contact: restitution of body %d must be in (0, 1]", b);
    c->contact = true;
    c->kc = contcoeff;
    c->resth.assign(restitution, restitution + nbodies);
    c->built = false;
    return TLSPH_OK;
}

tlsph_status tlsph_set_contact_friction(tlsph_ctx *c, int nbodies, const double *kfric) {
    if (!c) return TLSPH_ERR_ARG;
    if (!c->contact) return fail(c, TLSPH_ERR_STATE, "set_contact must come before set_contact_friction");
    if (nbodies != c->nspec || !kfric)
        return fail(c, TLSPH_ERR_ARG, "set_contact_friction: need one coefficient per specimen (%d)", c->nspec);
    bool any = false;
    for (int b = 0; b < nbodies; b++) {
        if (!(kfric[b] >= 0.0 && std::isfinite(kfric[b])))
            return fail(c, TLSPH_ERR_ARG, "set_contact_friction: coefficient of body %d must be finite and >= 0", b);
        any = any || kfric[b] > 0.0;
    }
    if (any) c->kfrich.assign(kfric, kfric + nbodies);
    else c->kfrich.clear();
    c->built = false;
    return TLSPH_OK;
}

tlsph_status tlsph_build_ref_neighbours(tlsph_ctx *c) {
    NvtxRange nv_("tlsph_build_ref_neighbours");
    DeviceScope ds_(c ? c->p.device : -1);
    if (!c) return TLSPH_ERR_ARG;
    if (c->n <= 0 || c->mats.empty()) return fail(c, TLSPH_ERR_STATE, "no particles");
    cudaSetDevice(c->p.device);
    tlsph_status st = c->p.precision == TLSPH_FP64 ? build_impl<double>(c) : build_impl<float>(c);
    if (st != TLSPH_OK && st != TLSPH_ERR_SINGULAR_L) free_device(c);
    return st;
}

tlsph_status tlsph_step_async(tlsph_ctx *c, int64_t nsteps) {
    NvtxRange nv_("tlsph_step");
    DeviceScope ds_(c ? c->p.device : -1);
    if (!c) return TLSPH_ERR_ARG;
    if (!c->built) return fail(c, TLSPH_ERR_STATE, "build_ref_neighbours must come before step");
    if (nsteps < 0) return fail(c, TLSPH_ERR_ARG, "negative step count");
    if (c->nexlist > 0 && c->ex_dirty) {
        tlsph_status st = ex_sync(c);
        if (st != TLSPH_OK) return st;
    }
    return c->p.precision == TLSPH_FP64 ? step_impl<double>(c, nsteps) : step_impl<float>(c, nsteps);
}

tlsph_status tlsph_sync(tlsph_ctx *c) {
    DeviceScope ds_(c ? c->p.device : -1);
    if (!c) return TLSPH_ERR_ARG;
    if (!c->built) return fail(c, TLSPH_ERR_STATE, "not built");
    return check_flags(c);
}

tlsph_status tlsph_step(tlsph_ctx *c, int64_t nsteps) {
    tlsph_status st = tlsph_step_async(c, nsteps);
    if (st != TLSPH_OK) return st;
    return check_flags(c);
}

int64_t tlsph_field_bytes(const tlsph_ctx *c, int field) {
    if (!c || c->n <= 0) return -1;
    if (field == TLSPH_FIELD_STATE) return c->built ? (int64_t)state_bytes(c) : -1;
    int nc = field_comps(c, field);
    return nc < 0 ? -1 : (int64_t)nc * c->n * 8;
}

tlsph_status tlsph_read_state(tlsph_ctx *c, int field, void *dst, size_t bytes, int dst_is_device) {
    DeviceScope ds_(c ? c->p.device : -1);
    if (!c) return TLSPH_ERR_ARG;
    if (!c->built) return fail(c, TLSPH_ERR_STATE, "build_ref_neighbours must come before read_state");
    int64_t need = tlsph_field_bytes(c, field);
    if (need < 0) return fail(c, TLSPH_ERR_ARG, "unknown field %d", field);
    if (!dst || bytes != (size_t)need) return fail(c, TLSPH_ERR_ARG, "read_state: need %lld bytes", (long long)need);
    if (field == TLSPH_FIELD_STATE) {
        if (dst_is_device) return fail(c, TLSPH_ERR_ARG, "the checkpoint blob is host memory");
        return c->p.precision == TLSPH_FP64 ? state_io<double>(c, (char *)dst, true)
                                            : state_io<float>(c, (char *)dst, true);
    }
    double *dev = (double *)dst;
    double *tmp = nullptr;
    if (!dst_is_device) {
        if (cudaMalloc(&tmp, need) != cudaSuccess) {
            cudaGetLastError();
            return fail(c, TLSPH_ERR_OOM, "read_state staging buffer");
        }
        dev = tmp;
    }
    tlsph_status st = c->p.precision == TLSPH_FP64 ? read_impl<double>(c, field, dev) : read_impl<float>(c, field, dev);
    if (st == TLSPH_OK && !dst_is_device) {
        cudaError_t e = cudaMemcpyAsync(dst, dev, need, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) st = fail(c, TLSPH_ERR_CUDA, "read_state copy: %s", cudaGetErrorString(e));
    } else if (st == TLSPH_OK) {
        cudaError_t e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) st = fail(c, TLSPH_ERR_CUDA, "read_state: %s", cudaGetErrorString(e));
    }
    if (tmp) cudaFree(tmp);
    return st;
}

tlsph_status tlsph_write_state(tlsph_ctx *c, int field, const void *src, size_t bytes, int src_is_device) {
    DeviceScope ds_(c ? c->p.device : -1);
    if (!c) return TLSPH_ERR_ARG;
    if (!c->built) return fail(c, TLSPH_ERR_STATE, "build_ref_neighbours must come before write_state");
    int64_t need = tlsph_field_bytes(c, field);
    if (need < 0) return fail(c, TLSPH_ERR_ARG, "unknown field %d", field);
    if (!src || bytes != (size_t)need) return fail(c, TLSPH_ERR_ARG, "write_state: need %lld bytes", (long long)need);
    if (field == TLSPH_FIELD_STATE) {
        if (src_is_device) return fail(c, TLSPH_ERR_ARG, "the checkpoint blob is host memory");
        return c->p.precision == TLSPH_FP64 ? state_io<double>(c, (char *)src, false)
                                            : state_io<float>(c, (char *)src, false);
    }
    const double *dev = (const double *)src;
    double *tmp = nullptr;
    if (!src_is_device) {
        if (cudaMalloc(&tmp, need) != cudaSuccess) {
            cudaGetLastError();
            return fail(c, TLSPH_ERR_OOM, "write_state staging buffer");
        }
        cudaMemcpyAsync(tmp, src, need, cudaMemcpyHostToDevice, c->stream);
        dev = tmp;
    }
    tlsph_status st =
        c->p.precision == TLSPH_FP64 ? write_impl<double>(c, field, dev) : write_impl<float>(c, field, dev);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (st == TLSPH_OK && e != cudaSuccess) st = fail(c, TLSPH_ERR_CUDA, "write_state: %s", cudaGetErrorString(e));
    if (tmp) cudaFree(tmp);
    return st;
}

tlsph_status tlsph_energies(tlsph_ctx *c, double out[6]) {
    DeviceScope ds_(c ? c->p.device : -1);
    if (!c || !out) return TLSPH_ERR_ARG;
    if (!c->built) return fail(c, TLSPH_ERR_STATE, "not built");
    return c->p.precision == TLSPH_FP64 ? energies_impl<double>(c, out) : energies_impl<float>(c, out);
}

tlsph_status tlsph_time(tlsph_ctx *c, int specimen, double *t, double *dt) {
    DeviceScope ds_(c ? c->p.device : -1);
    if (!c || !t || !dt) return TLSPH_ERR_ARG;
    if (!c->built) return fail(c, TLSPH_ERR_STATE, "not built");
    if (specimen < 0 || specimen >= c->nspec) return fail(c, TLSPH_ERR_ARG, "specimen out of range");
    CK(cudaMemcpyAsync(t, c->t + specimen, 8, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(dt, c->dt + specimen, 8, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return TLSPH_OK;
}

int64_t tlsph_nnz(const tlsph_ctx *c) { return (c && c->built) ? c->nnz : -1; }

tlsph_status tlsph_neighbours(tlsph_ctx *c, int64_t *row_ptr, int32_t *col, int64_t cap) {
    DeviceScope ds_(c ? c->p.device : -1);
    if (!c || !row_ptr || !col) return TLSPH_ERR_ARG;
    if (!c->built) return fail(c, TLSPH_ERR_STATE, "not built");
    if (cap < c->nnz) return fail(c, TLSPH_ERR_ARG, "cap < nnz (%lld)", (long long)c->nnz);
    const int64_t n = c->n;
    int64_t *len, *rp;
    int *co;
    size_t mark = c->allocs.size();
    DA(len, (n + 1) * 8);
    DA(rp, (n + 1) * 8);
    DA(co, std::max<int64_t>(c->nnz, 1) * 4);
    CK(cudaMemsetAsync(len, 0, (n + 1) * 8, c->stream));
    k_rowlen_caller<<<blocks_for(n), kThreads, 0, c->stream>>>(n, c->row_len, c->perm, len);
    CKL();
    tlsph_status st = scan_exclusive(c, n + 1, len, rp);
    if (st != TLSPH_OK) return st;
    k_rows_caller<<<blocks_for(n), kThreads, 0, c->stream>>>(n, c->row_ptr, c->col, c->perm, rp, co);
    CKL();
    CK(cudaMemcpyAsync(row_ptr, rp, (n + 1) * 8, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(col, co, c->nnz * 4, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    while (c->allocs.size() > mark) {
        cudaFree(c->allocs.back());
        c->mem_used -= c->alloc_bytes.back();
        c->alloc_bytes.pop_back();
        c->allocs.pop_back();
    }
    return TLSPH_OK;
}

tlsph_status tlsph_permutation(tlsph_ctx *c, int64_t *perm) {
    DeviceScope ds_(c ? c->p.device : -1);
    if (!c || !perm) return TLSPH_ERR_ARG;
    if (!c->built) return fail(c, TLSPH_ERR_STATE, "not built");
    std::vector<int> p(c->n);
    CK(cudaMemcpyAsync(p.data(), c->perm, c->n * 4, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    for (int64_t k = 0; k < c->n; k++) perm[k] = p[k];
    return TLSPH_OK;
}

tlsph_status tlsph_get_info(tlsph_ctx *c, tlsph_info *out) {
    DeviceScope ds_(c ? c->p.device : -1);
    if (!c || !out) return TLSPH_ERR_ARG;
    out->steps = c->steps;
    out->kernel_launches = c->launches;
    out->nnz = c->built ? c->nnz : -1;
    out->max_row = c->max_row;
    out->bytes_per_step = c->bytes_per_step;
    out->stencil = (c->layout != TLSPH_LAYOUT_CSR) ? c->nsten : 0;
    const bool lat = c->layout == TLSPH_LAYOUT_AUTO && c->lat_nx > 0;
    out->lattice_nx = lat ? c->lat_nx : 0;
    out->lattice_nxny = lat ? c->lat_nxny : 0;
    out->noconverge = out->nonfinite = 0;
    if (c->built) {
        int hf[kNumFlags];
        CK(cudaMemcpyAsync(hf, c->flags, sizeof hf, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        out->noconverge = hf[kFlagNoconv];
        out->nonfinite = hf[kFlagNonfinite];
    }
    return TLSPH_OK;
}

tlsph_status tlsph_set_option(tlsph_ctx *c, int option, int value) {
    DeviceScope ds_(c ? c->p.device : -1);
    if (!c) return TLSPH_ERR_ARG;
    if (option == TLSPH_OPT_KERNEL_TIMING) {
        if (c->timing && !value) {
            cudaStreamSynchronize(c->stream);
            collect_timing(c);
        }
        c->timing = value != 0;
        return TLSPH_OK;
    }
    if (option == TLSPH_OPT_RECORD_ACC) {
        c->record_acc = value != 0;
        drop_graph(c);
        return TLSPH_OK;
    }
    if (option == TLSPH_OPT_MODE) {
        if (value < TLSPH_MODE_LAUNCH || value > TLSPH_MODE_PERSISTENT) return fail(c, TLSPH_ERR_ARG, "bad mode");
        c->mode = value;
        drop_graph(c);
        return TLSPH_OK;
    }
    if (option == TLSPH_OPT_BLOCK) {
        if (value != 64 && value != 128 && value != 256) return fail(c, TLSPH_ERR_ARG, "block must be 64, 128 or 256");
        c->bs = value;
        drop_graph(c);
        return TLSPH_OK;
    }
    if (option == TLSPH_OPT_MEMORY_LIMIT) {
        if (value < 0) return fail(c, TLSPH_ERR_ARG, "memory limit must be >= 0 MiB");
        c->mem_limit = (size_t)value << 20;
        return TLSPH_OK;
    }
    if (option == TLSPH_OPT_BARRIER_TEST) {
        c->barrier_test = value != 0;
        return TLSPH_OK;
    }
    if (option == TLSPH_OPT_NEIGHBOUR_LAYOUT) {
        if (value != TLSPH_LAYOUT_AUTO && value != TLSPH_LAYOUT_CSR && value != TLSPH_LAYOUT_STENCIL)
            return fail(c, TLSPH_ERR_ARG, "bad layout");
        c->layout = value;
        drop_graph(c);
        return TLSPH_OK;
    }
    if (option == TLSPH_OPT_LATTICE_ROWS_GRADIENT || option == TLSPH_OPT_LATTICE_ROWS_FORCE) {
        if (value != 1 && value != 2 && !(value == 4 && option == TLSPH_OPT_LATTICE_ROWS_FORCE))
            return fail(c, TLSPH_ERR_ARG, "rows per thread must be 1 or 2 (or 4 in the force kernel)");
        (option == TLSPH_OPT_LATTICE_ROWS_GRADIENT ? c->lat_rows_grad : c->lat_rows_force) = value;
        drop_graph(c);
        return TLSPH_OK;
    }
    if (option == TLSPH_OPT_FUSE_STRESS) {
        c->fuse_stress = value != 0;
        drop_graph(c);
        return TLSPH_OK;
    }
    if (option == TLSPH_OPT_LATTICE_ZSTREAM) {
        if (value < 0) return fail(c, TLSPH_ERR_ARG, "planes per thread must be >= 0");
        c->lat_zc = value;
        drop_graph(c);
        return TLSPH_OK;
    }
    if (option == TLSPH_OPT_LATTICE_PATCH) {
        if (value != 0 && value != 32 && value != 64 && value != 128)
            return fail(c, TLSPH_ERR_ARG, "patch width must be 0, 32, 64 or 128");
        c->lat_cw = value;
        drop_graph(c);
        return TLSPH_OK;
    }
    return fail(c, TLSPH_ERR_ARG, "unknown option %d", option);
}

tlsph_status tlsph_autotune(tlsph_ctx *c, int trial_steps, tlsph_tuning *best, tlsph_tuning *all) {
    NvtxRange nv_("tlsph_autotune");
    DeviceScope ds_(c ? c->p.device : -1);
    if (!c) return TLSPH_ERR_ARG;
    if (!c->built) return fail(c, TLSPH_ERR_STATE, "build_ref_neighbours must come before autotune");
    if (trial_steps < 1) return fail(c, TLSPH_ERR_ARG, "trial_steps must be >= 1");
    return c->p.precision == TLSPH_FP64 ? autotune_impl<double>(c, trial_steps, best, all)
                                        : autotune_impl<float>(c, trial_steps, best, all);
}

tlsph_status tlsph_kernel_times(tlsph_ctx *c, double ms[3], int64_t count[3]) {
    DeviceScope ds_(c ? c->p.device : -1);
    if (!c || !ms || !count) return TLSPH_ERR_ARG;
    CK(cudaStreamSynchronize(c->stream));
    collect_timing(c);
    for (int q = 0; q < 3; q++) {
        ms[q] = c->ms[q];
        count[q] = c->cnt[q];
        c->ms[q] = 0.0;
        c->cnt[q] = 0;
    }
    return TLSPH_OK;
}

}  // extern "C"

// ===================================================================== allocation-free cell sort
// A variant of the reference setup's cell sort for callers that cannot allocate device
// memory (for example code that runs inside a memory pool it does not own, or a driver
// that forbids cudaMalloc while it holds the device).  Its scratch lives in one file-scope
// device array of fixed size, shared by every call on a device; nothing is allocated.
#include <mutex>

namespace {

constexpr int64_t kNAMax = TLSPH_NOALLOC_MAX_PARTICLES;
constexpr int64_t kNABlk = (kNAMax + kSortTile - 1) / kSortTile;

struct NAScratch {
    unsigned long long keys[2][kNAMax];
    int vals[2][kNAMax];
    int64_t hist[256 * kNABlk];
    int64_t hoff[256 * kNABlk];
    int64_t bsum[64];
    int64_t bscan[64];
    double bbox[8];  // min xyz, max xyz, specimens (largest id + 1), count of non-finite coordinates or negative ids
    CellGrid grid;
    int refused;     // inputs the context's reference setup refuses: every perm entry becomes -1
};

// every GPU that loads the library holds this array until the process exits
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NAScratch)];

std::mutex g_na_mutex;
void *g_na_ptr[128] = {nullptr};

__global__ void k_na_bbox(int64_t n, int dim, const double *X, const int32_t *spec, double *out) {
    __shared__ double smin[3][32], smax[3][32];
    __shared__ int sbad, sspec;
    if (threadIdx.x == 0) {
        sbad = 0;
        sspec = 0;
    }
    __syncthreads();
    double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    int bad = 0, smaxid = 0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        for (int k = 0; k < dim; k++) {
            double x = X[dim * i + k];
            bad += isfinite(x) ? 0 : 1;  // fmin / fmax below would drop a NaN silently
            mn[k] = fmin(mn[k], x);
            mx[k] = fmax(mx[k], x);
        }
        if (spec) {
            bad += spec[i] < 0 ? 1 : 0;
            smaxid = max(smaxid, spec[i]);
        }
    }
    if (bad) atomicAdd(&sbad, bad);
    atomicMax(&sspec, smaxid);
    for (int k = 0; k < 3; k++)
        for (int o = 16; o > 0; o >>= 1) {
            mn[k] = fmin(mn[k], __shfl_xor_sync(0xffffffffu, mn[k], o));
            mx[k] = fmax(mx[k], __shfl_xor_sync(0xffffffffu, mx[k], o));
        }
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0)
        for (int k = 0; k < 3; k++) {
            smin[k][w] = mn[k];
            smax[k][w] = mx[k];
        }
    __syncthreads();
    if (threadIdx.x == 0) {
        int nw = (blockDim.x + 31) >> 5;
        for (int k = 0; k < 3; k++) {
            double a = INFINITY, b = -INFINITY;
            for (int q = 0; q < nw; q++) {
                a = fmin(a, smin[k][q]);
                b = fmax(b, smax[k][q]);
            }
            if (k >= dim) a = b = 0.0;
            out[k] = a;
            out[3 + k] = b;
        }
        out[6] = (double)sspec + 1.0;
        out[7] = (double)sbad;
    }
}

// the same grid as the context's reference setup: cells R/3, nc = floor((max - min) / cs + 1/2) + 1, and the
// same refusals: a non-finite coordinate or negative specimen id, or keys (specimens x cells) of 9e18 or more
__global__ void k_na_grid(int dim, double cs, const double *bbox, CellGrid *g, int *refused) {
    g->dim = dim;
    g->cs = cs;
    bool ok = bbox[7] == 0.0;
    double maxkey = bbox[6];
    for (int k = 0; k < 3; k++) {
        g->xmin[k] = bbox[k];
        const double ncd = floor(__dadd_rn(__ddiv_rn(__dsub_rn(bbox[3 + k], bbox[k]), cs), 0.5)) + 1.0;
        ok = ok && isfinite(ncd);
        maxkey *= ncd;
        g->nc[k] = ok && ncd < 9.0e18 ? (int64_t)ncd : 1;
    }
    ok = ok && maxkey < 9.0e18;
    *refused = ok ? 0 : 1;
}

__global__ void k_na_keys(int64_t n, int dim, const double *X, const int32_t *spec, const CellGrid *gp,
                          const int *refused, unsigned long long *key, int *id) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    id[i] = (int)i;
    if (*refused) {  // the sort still runs on zero keys; k_na_copy writes -1
        key[i] = 0ull;
        return;
    }
    const CellGrid g = *gp;
    int64_t c[3] = {0, 0, 0};
    for (int k = 0; k < dim; k++) c[k] = cell_coord(X[dim * i + k], g.xmin[k], g.cs);
    int64_t sp = spec ? (int64_t)spec[i] : 0;
    key[i] = (unsigned long long)((((sp * g.nc[2] + c[2]) * g.nc[1] + c[1]) * g.nc[0]) + c[0]);
}

__global__ void k_na_copy(int64_t n, const int *src, const int *refused, int32_t *dst) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) dst[i] = *refused ? -1 : src[i];
}

}  // namespace

extern "C" tlsph_status tlsph_cell_sort_noalloc(int device, void *cuda_stream, int64_t n, int dim, double h,
                                                double support, const double *X0, const int32_t *specimen_id,
                                                int32_t *perm) {
    if (n < 1 || n > kNAMax || (dim != 2 && dim != 3) || !(h > 0.0) || !(support > 0.0) || !X0 || !perm ||
        device < 0 || device >= 128)
        return TLSPH_ERR_ARG;
    int prev = 0;
    if (cudaGetDevice(&prev) != cudaSuccess) {
        cudaGetLastError();
        return TLSPH_ERR_CUDA;
    }
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return TLSPH_ERR_CUDA;
    }
    tlsph_status st = TLSPH_OK;
    NAScratch *sc = nullptr;
    {
        // set-up, once per device, with that device current: the device address of the scratch
        std::lock_guard<std::mutex> lock(g_na_mutex);
        if (!g_na_ptr[device]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
                cudaGetLastError();
                st = TLSPH_ERR_CUDA;
            } else {
                g_na_ptr[device] = p;
            }
        }
        sc = reinterpret_cast<NAScratch *>(g_na_ptr[device]);
    }
    if (st == TLSPH_OK) {
        cudaStream_t s = (cudaStream_t)cuda_stream;
        const int64_t nblk = (n + kSortTile - 1) / kSortTile;
        const int64_t m = 256 * nblk;
        const unsigned nb = (unsigned)((m + kScanBlock - 1) / kScanBlock);
        k_na_bbox<<<1, 1024, 0, s>>>(n, dim, X0, specimen_id, sc->bbox);
        k_na_grid<<<1, 1, 0, s>>>(dim, support * h / 3.0, sc->bbox, &sc->grid, &sc->refused);
        k_na_keys<<<blocks_for(n), kThreads, 0, s>>>(n, dim, X0, specimen_id, &sc->grid, &sc->refused, sc->keys[0],
                                                     sc->vals[0]);
        // stable LSD radix sort over all 64 key bits: 8 passes, the result lands in buffer 0
        for (int pass = 0; pass < 8; pass++) {
            const int cur = pass & 1, shift = 8 * pass;
            k_radix_hist<<<(unsigned)nblk, 32, 0, s>>>(n, sc->keys[cur], shift, sc->hist);
            k_scan_block<<<nb, kScanBlock, 0, s>>>(m, sc->hist, sc->hoff, sc->bsum);
            k_scan_block<<<1, kScanBlock, 0, s>>>((int64_t)nb, sc->bsum, sc->bscan, nullptr);
            k_scan_add<<<nb, kScanBlock, 0, s>>>(m, sc->hoff, sc->bscan);
            k_radix_scatter<<<(unsigned)nblk, 32, 0, s>>>(n, sc->keys[cur], sc->vals[cur], shift, sc->hoff,
                                                          sc->keys[cur ^ 1], sc->vals[cur ^ 1]);
        }
        k_na_copy<<<blocks_for(n), kThreads, 0, s>>>(n, sc->vals[0], &sc->refused, perm);
        if (cudaGetLastError() != cudaSuccess) st = TLSPH_ERR_CUDA;
    }
    cudaSetDevice(prev);
    return st;
}


// ===================================================================== learned constitutive surrogate
struct tlsph_mlp {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int batch = 0;
    std::string err;
    std::vector<void *> allocs;
    float *P = nullptr, *G = nullptr, *m = nullptr, *v = nullptr;  // master parameters, gradient, Adam moments
    __nv_bfloat16 *Wb = nullptr, *W1T = nullptr, *W2T = nullptr, *W3T = nullptr;
    float *biasc = nullptr, *norm = nullptr;
    __nv_bfloat16 *Xb, *A0, *A1, *A2, *dZb, *dZT, *AT, *XbT, *doutb, *doutT;
    float *Yn, *Z0, *Z1, *Z2, *out, *dout, *dA, *dZf, *loss;
    double *stat_d;
    float *stat_f;
    int *tc_flag;           // tensor-core waits that ran out in the last forward
    int *gemm_flag;         // tensor-core waits of the training GEMMs that ran out (cleared when reported)
    int tensor_path = TLSPH_TENSOR_TCGEN05;
    int64_t t = 0;
};

namespace {

tlsph_status mfail(tlsph_mlp *m, tlsph_status st, const char *msg) {
    if (m) m->err = msg;
    return st;
}
#define MK(call)                                                                  \
    do {                                                                          \
        cudaError_t e_ = (call);                                                  \
        if (e_ != cudaSuccess) return mfail(m, TLSPH_ERR_CUDA, cudaGetErrorString(e_)); \
    } while (0)

template <typename P> tlsph_status malloc_m(tlsph_mlp *m, P **ptr, size_t bytes) {
    void *q = nullptr;
    if (cudaMalloc(&q, bytes ? bytes : 16) != cudaSuccess) {
        cudaGetLastError();
        return mfail(m, TLSPH_ERR_OOM, "cudaMalloc");
    }
    m->allocs.push_back(q);
    *ptr = reinterpret_cast<P *>(q);
    return TLSPH_OK;
}
#define MA(ptr, bytes)                                     \
    do {                                                   \
        tlsph_status s_ = malloc_m(m, &(ptr), (bytes));    \
        if (s_ != TLSPH_OK) return s_;                     \
    } while (0)

inline unsigned nblk(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// refresh the bf16 weights, their transposes and the contiguous biases from the master copy
tlsph_status mlp_refresh(tlsph_mlp *m) {
    cudaStream_t s = m->stream;
    k_f32_to_bf16<<<nblk(kHid * kIn), 256, 0, s>>>(kHid * kIn, m->P + kOffW0, m->Wb);
    k_f32_to_bf16<<<nblk(kHid * kHid), 256, 0, s>>>(kHid * kHid, m->P + kOffW1, m->Wb + kHid * kIn);
    k_f32_to_bf16<<<nblk(kHid * kHid), 256, 0, s>>>(kHid * kHid, m->P + kOffW2, m->Wb + kHid * kIn + kHid * kHid);
    k_f32_to_bf16<<<nblk(kOut * kHid), 256, 0, s>>>(kOut * kHid, m->P + kOffW3,
                                                   m->Wb + kHid * kIn + 2 * kHid * kHid);
    const dim3 tb(32, 8);
    k_transpose_bf16<<<dim3(kHid / 32, kHid / 32), tb, 0, s>>>(kHid, kHid, m->Wb + kHid * kIn, m->W1T);
    k_transpose_bf16<<<dim3(kHid / 32, kHid / 32), tb, 0, s>>>(kHid, kHid, m->Wb + kHid * kIn + kHid * kHid, m->W2T);
    k_transpose_bf16<<<dim3(kHid / 32, 1), tb, 0, s>>>(kOut, kHid, m->Wb + kHid * kIn + 2 * kHid * kHid, m->W3T);
    MK(cudaMemcpyAsync(m->biasc, m->P + kOffB0, kHid * 4, cudaMemcpyDeviceToDevice, s));
    MK(cudaMemcpyAsync(m->biasc + kHid, m->P + kOffB1, kHid * 4, cudaMemcpyDeviceToDevice, s));
    MK(cudaMemcpyAsync(m->biasc + 2 * kHid, m->P + kOffB2, kHid * 4, cudaMemcpyDeviceToDevice, s));
    MK(cudaMemcpyAsync(m->biasc + 3 * kHid, m->P + kOffB3, kOut * 4, cudaMemcpyDeviceToDevice, s));
    MK(cudaGetLastError());
    return TLSPH_OK;
}

// The training GEMMs on the network's tensor path: tcgen05 (k_gemm_tc, one CTA per 128 x 128 output tile)
// or warp-level mma.sync (k_gemm_bf16).
template <int EPI>
void gemm(tlsph_mlp *m, int M, int N, int K, const __nv_bfloat16 *A, const __nv_bfloat16 *B, const float *bias,
          float *C, __nv_bfloat16 *Aout) {
    if (m->tensor_path == TLSPH_TENSOR_TCGEN05) {
        const dim3 grid((unsigned)((M + 127) / 128), (unsigned)((N + 127) / 128));
        k_gemm_tc<EPI><<<grid, 128, sizeof(GemmTcSmem), m->stream>>>(M, N, K, A, B, bias, C, Aout, m->gemm_flag);
        return;
    }
    const int warps = (M / 16) * ((N + 31) / 32);
    k_gemm_bf16<EPI><<<(unsigned)((warps + 3) / 4), 128, 0, m->stream>>>(M, N, K, A, B, bias, C, Aout);
}
// TLSPH_ERR_TIMEOUT (and the flag cleared) when a training GEMM's wait on the tensor cores ran out; the
// stream must be synchronised.
tlsph_status gemm_check(tlsph_mlp *m) {
    int h = 0;
    MK(cudaMemcpy(&h, m->gemm_flag, sizeof h, cudaMemcpyDeviceToHost));
    if (!h) return TLSPH_OK;
    MK(cudaMemset(m->gemm_flag, 0, sizeof h));
    return mfail(m, TLSPH_ERR_TIMEOUT, "a tensor-core wait of a training GEMM ran out");
}
void transpose(tlsph_mlp *m, int rows, int cols, const __nv_bfloat16 *in, __nv_bfloat16 *out) {
    k_transpose_bf16<<<dim3((cols + 31) / 32, (rows + 31) / 32), dim3(32, 8), 0, m->stream>>>(rows, cols, in, out);
}

// forward + backward of one batch of raw rows; gradients into m->G, loss into m->loss
tlsph_status mlp_fwd_bwd(tlsph_mlp *m, const float *x, const float *y) {
    const int B = m->batch;
    cudaStream_t s = m->stream;
    const float *nm = m->norm;
    k_normalize<<<nblk((int64_t)B * 16), 256, 0, s>>>(B, x, nm, nm + 16, nullptr, m->Xb);
    k_normalize<<<nblk((int64_t)B * 16), 256, 0, s>>>(B, y, nm + 32, nm + 48, m->Yn, nullptr);
    const __nv_bfloat16 *W0 = m->Wb, *W1 = m->Wb + kHid * kIn, *W2 = W1 + kHid * kHid, *W3 = W2 + kHid * kHid;
    gemm<1>(m, B, kHid, kIn, m->Xb, W0, m->biasc, m->Z0, m->A0);
    gemm<1>(m, B, kHid, kHid, m->A0, W1, m->biasc + kHid, m->Z1, m->A1);
    gemm<1>(m, B, kHid, kHid, m->A1, W2, m->biasc + 2 * kHid, m->Z2, m->A2);
    gemm<0>(m, B, kOut, kHid, m->A2, W3, m->biasc + 3 * kHid, m->out, nullptr);
    MK(cudaMemsetAsync(m->loss, 0, 4, s));
    k_mse_grad<<<nblk((int64_t)B * kOut), 256, 0, s>>>((int64_t)B * kOut, m->out, m->Yn, m->dout, m->doutb, m->loss);
    // layer 3
    transpose(m, B, kOut, m->doutb, m->doutT);
    transpose(m, B, kHid, m->A2, m->AT);
    gemm<0>(m, kOut, kHid, B, m->doutT, m->AT, nullptr, m->G + kOffW3, nullptr);
    k_colsum<<<kOut, 256, 0, s>>>(B, kOut, m->dout, m->G + kOffB3);
    gemm<0>(m, B, kHid, kOut, m->doutb, m->W3T, nullptr, m->dA, nullptr);
    // layers 2, 1, 0
    const float *Zs[3] = {m->Z0, m->Z1, m->Z2};
    const __nv_bfloat16 *Ain[3] = {m->Xb, m->A0, m->A1};
    const __nv_bfloat16 *WT[3] = {nullptr, m->W1T, m->W2T};
    const int offW[3] = {kOffW0, kOffW1, kOffW2}, offB[3] = {kOffB0, kOffB1, kOffB2}, nin[3] = {kIn, kHid, kHid};
    for (int l = 2; l >= 0; l--) {
        k_silu_back_f32<<<nblk((int64_t)B * kHid), 256, 0, s>>>((int64_t)B * kHid, m->dA, Zs[l], m->dZf);
        k_f32_to_bf16<<<nblk((int64_t)B * kHid), 256, 0, s>>>((int64_t)B * kHid, m->dZf, m->dZb);
        transpose(m, B, kHid, m->dZb, m->dZT);
        transpose(m, B, nin[l], Ain[l], l == 0 ? m->XbT : m->AT);
        gemm<0>(m, kHid, nin[l], B, m->dZT, l == 0 ? m->XbT : m->AT, nullptr, m->G + offW[l], nullptr);
        k_colsum<<<kHid, 256, 0, s>>>(B, kHid, m->dZf, m->G + offB[l]);
        if (l > 0) gemm<0>(m, B, kHid, kHid, m->dZb, WT[l], nullptr, m->dA, nullptr);
    }
    MK(cudaGetLastError());
    return TLSPH_OK;
}

}  // namespace

extern "C" {

tlsph_status tlsph_mlp_create(int device, void *cuda_stream, int batch, tlsph_mlp **out) {
    if (!out) return TLSPH_ERR_ARG;
    *out = nullptr;
    if (batch < 16 || batch % 16 || batch > (1 << 20)) return TLSPH_ERR_ARG;
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return TLSPH_ERR_CUDA;
    }
    tlsph_mlp *m = new tlsph_mlp();
    m->device = device;
    m->batch = batch;
    if (cuda_stream) m->stream = (cudaStream_t)cuda_stream;
    else if (cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking) == cudaSuccess) m->own_stream = true;
    const size_t B = (size_t)batch;
    tlsph_status st = TLSPH_OK;
#define MAX(ptr, bytes)                          \
    if (st == TLSPH_OK) st = malloc_m(m, &(ptr), (bytes));
    MAX(m->P, kNumParams * 4) MAX(m->G, kNumParams * 4) MAX(m->m, kNumParams * 4) MAX(m->v, kNumParams * 4)
    MAX(m->Wb, kNumWeights * 2) MAX(m->W1T, kHid * kHid * 2) MAX(m->W2T, kHid * kHid * 2) MAX(m->W3T, kHid * kOut * 2)
    MAX(m->biasc, (3 * kHid + kOut) * 4) MAX(m->norm, 96 * 4)
    MAX(m->Xb, B * kIn * 2) MAX(m->A0, B * kHid * 2) MAX(m->A1, B * kHid * 2) MAX(m->A2, B * kHid * 2)
    MAX(m->dZb, B * kHid * 2) MAX(m->dZT, B * kHid * 2) MAX(m->AT, B * kHid * 2) MAX(m->XbT, B * kIn * 2)
    MAX(m->doutb, B * kOut * 2) MAX(m->doutT, B * kOut * 2)
    MAX(m->Yn, B * kOut * 4) MAX(m->Z0, B * kHid * 4) MAX(m->Z1, B * kHid * 4) MAX(m->Z2, B * kHid * 4)
    MAX(m->out, B * kOut * 4) MAX(m->dout, B * kOut * 4) MAX(m->dA, B * kHid * 4) MAX(m->dZf, B * kHid * 4)
    MAX(m->loss, 4) MAX(m->stat_d, 64 * 8) MAX(m->stat_f, 64 * 4) MAX(m->tc_flag, 4) MAX(m->gemm_flag, 4)
#undef MAX
    if (st != TLSPH_OK) {
        tlsph_mlp_destroy(m);
        return st;
    }
    cudaMemsetAsync(m->gemm_flag, 0, sizeof(int), m->stream);
    if (cudaFuncSetAttribute(k_gemm_tc<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(GemmTcSmem)) !=
            cudaSuccess ||
        cudaFuncSetAttribute(k_gemm_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(GemmTcSmem)) !=
            cudaSuccess ||
        cudaFuncSetAttribute(k_gemm_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(GemmTcSmem)) !=
            cudaSuccess) {
        cudaGetLastError();
        tlsph_mlp_destroy(m);
        return TLSPH_ERR_CUDA;
    }
    cudaMemsetAsync(m->P, 0, kNumParams * 4, m->stream);
    cudaMemsetAsync(m->m, 0, kNumParams * 4, m->stream);
    cudaMemsetAsync(m->v, 0, kNumParams * 4, m->stream);
    std::vector<float> nrm(96, 0.0f);
    for (int c = 0; c < 16; c++) {
        nrm[16 + c] = 1.0f;
        nrm[48 + c] = 1.0f;
        nrm[64 + c] = -INFINITY;
        nrm[80 + c] = INFINITY;
    }
    cudaMemcpyAsync(m->norm, nrm.data(), 96 * 4, cudaMemcpyHostToDevice, m->stream);
    st = mlp_refresh(m);
    if (st == TLSPH_OK && cudaStreamSynchronize(m->stream) != cudaSuccess) st = TLSPH_ERR_CUDA;
    if (st != TLSPH_OK) {
        tlsph_mlp_destroy(m);
        return st;
    }
    *out = m;
    return TLSPH_OK;
}

void tlsph_mlp_destroy(tlsph_mlp *m) {
    if (!m) return;
    cudaSetDevice(m->device);
    if (m->stream) cudaStreamSynchronize(m->stream);
    for (void *q : m->allocs) cudaFree(q);
    if (m->own_stream) cudaStreamDestroy(m->stream);
    delete m;
}

const char *tlsph_mlp_last_error(const tlsph_mlp *m) { return m ? m->err.c_str() : "null network"; }

tlsph_status tlsph_mlp_set_params(tlsph_mlp *m, const float *params) {
    DeviceScope ds_(m ? m->device : -1);
    if (!m || !params) return TLSPH_ERR_ARG;
    MK(cudaMemcpyAsync(m->P, params, kNumParams * 4, cudaMemcpyHostToDevice, m->stream));
    MK(cudaMemsetAsync(m->m, 0, kNumParams * 4, m->stream));
    MK(cudaMemsetAsync(m->v, 0, kNumParams * 4, m->stream));
    m->t = 0;
    tlsph_status st = mlp_refresh(m);
    if (st != TLSPH_OK) return st;
    MK(cudaStreamSynchronize(m->stream));
    return TLSPH_OK;
}

tlsph_status tlsph_mlp_get_params(tlsph_mlp *m, float *params) {
    DeviceScope ds_(m ? m->device : -1);
    if (!m || !params) return TLSPH_ERR_ARG;
    MK(cudaMemcpyAsync(params, m->P, kNumParams * 4, cudaMemcpyDeviceToHost, m->stream));
    MK(cudaStreamSynchronize(m->stream));
    return TLSPH_OK;
}

tlsph_status tlsph_mlp_set_normalization(tlsph_mlp *m, const float norm[96]) {
    DeviceScope ds_(m ? m->device : -1);
    if (!m || !norm) return TLSPH_ERR_ARG;
    for (int c = 0; c < 16; c++)
        if (!(norm[16 + c] > 0.0f) || !(norm[48 + c] > 0.0f)) return mfail(m, TLSPH_ERR_ARG, "std must be > 0");
    MK(cudaMemcpyAsync(m->norm, norm, 96 * 4, cudaMemcpyHostToDevice, m->stream));
    MK(cudaStreamSynchronize(m->stream));
    return TLSPH_OK;
}

tlsph_status tlsph_mlp_get_normalization(tlsph_mlp *m, float norm[96]) {
    DeviceScope ds_(m ? m->device : -1);
    if (!m || !norm) return TLSPH_ERR_ARG;
    MK(cudaMemcpyAsync(norm, m->norm, 96 * 4, cudaMemcpyDeviceToHost, m->stream));
    MK(cudaStreamSynchronize(m->stream));
    return TLSPH_OK;
}

tlsph_status tlsph_mlp_fit_normalization(tlsph_mlp *m, int64_t n, const float *x, const float *y, float margin) {
    DeviceScope ds_(m ? m->device : -1);
    if (!m || !x || !y || n < 2 || !(margin >= 0.0f)) return TLSPH_ERR_ARG;
    cudaStream_t s = m->stream;
    float st_h[6][16];
    double mean[2][16], sd[2][16];
    for (int which = 0; which < 2; which++) {
        MK(cudaMemsetAsync(m->stat_d, 0, 32 * 8, s));
        std::vector<float> init(32);
        for (int c = 0; c < 16; c++) {
            init[c] = INFINITY;
            init[16 + c] = -INFINITY;
        }
        // the ordered-int encoding of the min / max starts from +inf / -inf
        std::vector<int> enc(32);
        for (int c = 0; c < 32; c++) {
            int b;
            memcpy(&b, &init[c], 4);
            enc[c] = b < 0 ? (int)(0x80000000u - (unsigned)b) : b;
        }
        MK(cudaMemcpyAsync(m->stat_f, enc.data(), 32 * 4, cudaMemcpyHostToDevice, s));
        k_col_stats<<<dim3(64, 16), 256, 0, s>>>(n, which ? y : x, m->stat_d, m->stat_d + 16, m->stat_f,
                                                  m->stat_f + 16);
        MK(cudaGetLastError());
        double sums[32];
        int mm[32];
        MK(cudaMemcpyAsync(sums, m->stat_d, 32 * 8, cudaMemcpyDeviceToHost, s));
        MK(cudaMemcpyAsync(mm, m->stat_f, 32 * 4, cudaMemcpyDeviceToHost, s));
        MK(cudaStreamSynchronize(s));
        for (int c = 0; c < 16; c++) {
            const double mu = sums[c] / (double)n;
            double var = sums[16 + c] / (double)n - mu * mu;
            if (var < 0.0) var = 0.0;
            double sdev = sqrt(var);
            if (!(sdev > 1e-12 * std::max(1.0, fabs(mu)))) sdev = std::max(1.0, fabs(mu)) * 1e-6;
            mean[which][c] = mu;
            sd[which][c] = sdev;
            if (which == 0) {
                float lo, hi;
                int a = mm[c], b = mm[16 + c];
                if (a < 0) a = (int)(0x80000000u - (unsigned)a);
                if (b < 0) b = (int)(0x80000000u - (unsigned)b);
                memcpy(&lo, &a, 4);
                memcpy(&hi, &b, 4);
                const double nlo = (lo - mu) / sdev, nhi = (hi - mu) / sdev, w = nhi - nlo;
                st_h[4][c] = (float)(nlo - margin * w);
                st_h[5][c] = (float)(nhi + margin * w);
            }
        }
    }
    for (int c = 0; c < 16; c++) {
        st_h[0][c] = (float)mean[0][c];
        st_h[1][c] = (float)sd[0][c];
        st_h[2][c] = (float)mean[1][c];
        st_h[3][c] = (float)sd[1][c];
    }
    MK(cudaMemcpyAsync(m->norm, st_h, 96 * 4, cudaMemcpyHostToDevice, s));
    MK(cudaStreamSynchronize(s));
    return TLSPH_OK;
}

tlsph_status tlsph_mlp_gradients(tlsph_mlp *m, const float *x, const float *y, float *grads, float *loss) {
    DeviceScope ds_(m ? m->device : -1);
    if (!m || !x || !y) return TLSPH_ERR_ARG;
    tlsph_status st = mlp_fwd_bwd(m, x, y);
    if (st != TLSPH_OK) return st;
    if (grads) MK(cudaMemcpyAsync(grads, m->G, kNumParams * 4, cudaMemcpyDeviceToHost, m->stream));
    if (loss) MK(cudaMemcpyAsync(loss, m->loss, 4, cudaMemcpyDeviceToHost, m->stream));
    MK(cudaStreamSynchronize(m->stream));
    return gemm_check(m);
}

tlsph_status tlsph_mlp_train_step(tlsph_mlp *m, const float *x, const float *y, float lr, float *loss) {
    DeviceScope ds_(m ? m->device : -1);
    if (!m || !x || !y || !(lr > 0.0f)) return TLSPH_ERR_ARG;
    tlsph_status st = mlp_fwd_bwd(m, x, y);
    if (st != TLSPH_OK) return st;
    m->t++;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - powf(b1, (float)m->t), c2 = 1.0f - powf(b2, (float)m->t);
    k_adam<<<nblk(kNumParams), 256, 0, m->stream>>>(kNumParams, m->P, m->G, m->m, m->v, lr, b1, b2, 1e-8f, c1, c2);
    MK(cudaGetLastError());
    st = mlp_refresh(m);
    if (st != TLSPH_OK) return st;
    if (loss) {
        MK(cudaMemcpyAsync(loss, m->loss, 4, cudaMemcpyDeviceToHost, m->stream));
        MK(cudaStreamSynchronize(m->stream));
        return gemm_check(m);
    }
    return TLSPH_OK;
}

tlsph_status tlsph_mlp_forward(tlsph_mlp *m, int64_t n, const float *x, float *y, int32_t *outside) {
    DeviceScope ds_(m ? m->device : -1);
    if (!m || !x || !y || n < 1) return TLSPH_ERR_ARG;
    SurrogateDev d{};
    d.W = m->Wb;
    d.bias = m->biasc;
    d.in_mean = m->norm;
    d.in_std = m->norm + 16;
    d.out_mean = m->norm + 32;
    d.out_std = m->norm + 48;
    d.env_lo = m->norm + 64;
    d.env_hi = m->norm + 80;
    d.enabled = 1;
    if (m->tensor_path == TLSPH_TENSOR_TCGEN05) {
        MK(cudaFuncSetAttribute(k_mlp_forward_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(MlpTcSmem)));
        int nsm = 0, per_sm = 0;
        MK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, m->device));
        MK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mlp_forward_tc, 128 * kTcGroups, sizeof(MlpTcSmem)));
        const int64_t ctas = (n + 128 * kTcGroups - 1) / (128 * kTcGroups);
        const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((int64_t)std::max(per_sm, 1) * nsm, ctas));
        MK(cudaMemsetAsync(m->tc_flag, 0, sizeof(int), m->stream));
        k_mlp_forward_tc<<<grid, 128 * kTcGroups, sizeof(MlpTcSmem), m->stream>>>(n, x, y, d, outside, m->tc_flag);
        MK(cudaGetLastError());
        int h = 0;
        MK(cudaMemcpyAsync(&h, m->tc_flag, sizeof h, cudaMemcpyDeviceToHost, m->stream));
        MK(cudaStreamSynchronize(m->stream));
        if (h) return mfail(m, TLSPH_ERR_TIMEOUT, "a tensor-core wait ran out");
        return TLSPH_OK;
    }
    MK(cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(MlpSmem)));
    k_mlp_forward<<<(unsigned)((n + 127) / 128), 128, sizeof(MlpSmem), m->stream>>>(n, x, y, d, outside);
    MK(cudaGetLastError());
    MK(cudaStreamSynchronize(m->stream));
    return TLSPH_OK;
}

tlsph_status tlsph_mlp_set_tensor_path(tlsph_mlp *m, int path) {
    if (!m) return TLSPH_ERR_ARG;
    if (path != TLSPH_TENSOR_MMA_SYNC && path != TLSPH_TENSOR_TCGEN05) return mfail(m, TLSPH_ERR_ARG, "unknown tensor path");
    m->tensor_path = path;
    return TLSPH_OK;
}

tlsph_status tlsph_set_surrogate(tlsph_ctx *c, const tlsph_mlp *m, int scope) {
    DeviceScope ds_(c ? c->p.device : -1);
    if (!c) return TLSPH_ERR_ARG;
    if (!c->built) return fail(c, TLSPH_ERR_STATE, "build_ref_neighbours must come before set_surrogate");
    if (!m) {
        c->sur_on = false;
        return TLSPH_OK;
    }
    if (scope != TLSPH_SURROGATE_ALL && scope != TLSPH_SURROGATE_PLASTIC)
        return fail(c, TLSPH_ERR_ARG, "unknown surrogate scope %d", scope);
    if (c->p.precision != TLSPH_FP32_U64) return fail(c, TLSPH_ERR_ARG, "the surrogate runs in the FP32 step only");
    if (!c->sur_W) {
        DA(c->sur_W, kNumWeights * 2);
        DA(c->sur_bias, (3 * kHid + kOut) * 4);
        DA(c->sur_norm, 96 * 4);
        DA(c->sur_count, 3 * sizeof(unsigned long long));
        DA(c->sur_exact, c->n * sizeof(int));
        DA(c->sur_nexact, sizeof(unsigned));
    }
    CK(cudaStreamSynchronize(m->stream));
    CK(cudaMemcpyAsync(c->sur_W, m->Wb, kNumWeights * 2, cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaMemcpyAsync(c->sur_bias, m->biasc, (3 * kHid + kOut) * 4, cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaMemcpyAsync(c->sur_norm, m->norm, 96 * 4, cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaMemsetAsync(c->sur_count, 0, 3 * sizeof(unsigned long long), c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->sur_on = true;
    c->sur_scope = scope;
    c->sur_tensor = m->tensor_path;
    c->mode = TLSPH_MODE_LAUNCH;
    drop_graph(c);
    return TLSPH_OK;
}

// Network file: 8-byte magic "TLSPHMLP", uint32 version (1), uint32 parameter count, uint32 normalisation
// count (96), then the FP32 master parameters and the normalisation table, little-endian.
tlsph_status tlsph_mlp_save(tlsph_mlp *m, const char *path) {
    if (!m || !path) return TLSPH_ERR_ARG;
    std::vector<float> P(kNumParams), N(96);
    tlsph_status st = tlsph_mlp_get_params(m, P.data());
    if (st != TLSPH_OK) return st;
    st = tlsph_mlp_get_normalization(m, N.data());
    if (st != TLSPH_OK) return st;
    FILE *f = fopen(path, "wb");
    if (!f) return mfail(m, TLSPH_ERR_ARG, "cannot open the file for writing");
    const uint32_t hdr[3] = {1u, (uint32_t)kNumParams, 96u};
    bool ok = fwrite("TLSPHMLP", 1, 8, f) == 8 && fwrite(hdr, 4, 3, f) == 3 &&
              fwrite(P.data(), 4, P.size(), f) == P.size() && fwrite(N.data(), 4, N.size(), f) == N.size();
    ok = (fclose(f) == 0) && ok;
    return ok ? TLSPH_OK : mfail(m, TLSPH_ERR_ARG, "writing the network file failed");
}

tlsph_status tlsph_mlp_load(tlsph_mlp *m, const char *path) {
    if (!m || !path) return TLSPH_ERR_ARG;
    FILE *f = fopen(path, "rb");
    if (!f) return mfail(m, TLSPH_ERR_ARG, "cannot open the network file");
    char magic[8];
    uint32_t hdr[3];
    std::vector<float> P(kNumParams), N(96);
    bool ok = fread(magic, 1, 8, f) == 8 && memcmp(magic, "TLSPHMLP", 8) == 0 && fread(hdr, 4, 3, f) == 3 &&
              hdr[0] == 1u && hdr[1] == (uint32_t)kNumParams && hdr[2] == 96u &&
              fread(P.data(), 4, P.size(), f) == P.size() && fread(N.data(), 4, N.size(), f) == N.size();
    fclose(f);
    if (!ok) return mfail(m, TLSPH_ERR_ARG, "not a network file of this layout (16-128-128-128-16)");
    tlsph_status st = tlsph_mlp_set_params(m, P.data());
    if (st != TLSPH_OK) return st;
    return tlsph_mlp_set_normalization(m, N.data());
}

tlsph_status tlsph_load_surrogate(tlsph_ctx *c, const char *path, int scope) {
    DeviceScope ds_(c ? c->p.device : -1);
    if (!c) return TLSPH_ERR_ARG;
    if (!path) return fail(c, TLSPH_ERR_ARG, "load_surrogate: null path");
    tlsph_mlp *m = nullptr;
    tlsph_status st = tlsph_mlp_create(c->p.device, c->stream, 256, &m);
    if (st != TLSPH_OK) return fail(c, st, "load_surrogate: cannot create the network");
    st = tlsph_mlp_load(m, path);
    if (st != TLSPH_OK) {
        fail(c, st, "load_surrogate: %s", m->err.c_str());
        tlsph_mlp_destroy(m);
        return st;
    }
    st = tlsph_set_surrogate(c, m, scope);
    tlsph_mlp_destroy(m);
    return st;
}

tlsph_status tlsph_surrogate_counts(tlsph_ctx *c, int64_t counts[3]) {
    DeviceScope ds_(c ? c->p.device : -1);
    if (!c || !counts) return TLSPH_ERR_ARG;
    unsigned long long h[3] = {0, 0, 0};
    if (c->sur_count) {
        CK(cudaMemcpyAsync(h, c->sur_count, sizeof h, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
    }
    for (int q = 0; q < 3; q++) counts[q] = (int64_t)h[q];
    return TLSPH_OK;
}

tlsph_status tlsph_j2_samples(tlsph_ctx *c, int stride_elastic, int stride_plastic, unsigned salt, float *x,
                              float *y, float *pnorm, int64_t cap, int64_t *count) {
    DeviceScope ds_(c ? c->p.device : -1);
    if (!c || !x || !y || !count || cap < 0 || stride_elastic < 1 || stride_plastic < 1) return TLSPH_ERR_ARG;
    if (!c->built) return fail(c, TLSPH_ERR_STATE, "not built");
    const int64_t n = c->n;
    int64_t *flag, *off;
    size_t mark = c->allocs.size();
    DA(flag, (n + 1) * sizeof(int64_t));
    DA(off, (n + 1) * sizeof(int64_t));
    CK(cudaMemsetAsync(flag + n, 0, sizeof(int64_t), c->stream));
    const unsigned nb = blocks_for(n);
    auto run = [&](auto tag, auto dimc) -> tlsph_status {
        using T = decltype(tag);
        constexpr int D = decltype(dimc)::value;
        StepArgs<T> a = make_args<T>(c);
        k_gradient<T, D, false, false, kThreads><<<nb, kThreads, 0, c->stream>>>(a);
        CKL();
        k_j2_samples<T, D, false><<<nb, kThreads, 0, c->stream>>>(a, stride_elastic, stride_plastic, salt, flag,
                                                                   nullptr, x, y, pnorm, cap);
        CKL();
        tlsph_status st = scan_exclusive(c, n + 1, flag, off);
        if (st != TLSPH_OK) return st;
        k_j2_samples<T, D, true><<<nb, kThreads, 0, c->stream>>>(a, stride_elastic, stride_plastic, salt, flag, off,
                                                                  x, y, pnorm, cap);
        CKL();
        return TLSPH_OK;
    };
    tlsph_status st;
    if (c->p.precision == TLSPH_FP64)
        st = c->p.dim == 3 ? run(double(), std::integral_constant<int, 3>()) : run(double(), std::integral_constant<int, 2>());
    else
        st = c->p.dim == 3 ? run(float(), std::integral_constant<int, 3>()) : run(float(), std::integral_constant<int, 2>());
    if (st != TLSPH_OK) return st;
    int64_t h = 0;
    CK(cudaMemcpyAsync(&h, off + n, sizeof h, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    *count = std::min<int64_t>(h, cap);
    while (c->allocs.size() > mark) {
        cudaFree(c->allocs.back());
        c->mem_used -= c->alloc_bytes.back();
        c->alloc_bytes.pop_back();
        c->allocs.pop_back();
    }
    return TLSPH_OK;
}

}  // extern "C"
