// C ABI of libdgw: contexts, argument checks, launch sequences, CUDA-graph replay of
// the SSP-RK3 loop, projection and the mass diagnostic.  See include/dgw.h.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <set>
#include <string>
#include <tuple>
#include <vector>
#include <algorithm>
#include <vector>
#include <algorithm>
#include <numeric>

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include "../../include/dgw.h"
#include "dgw_internal.h"
#include "dgw_math.cuh"

using namespace dgw;

static thread_local std::string g_err;

static dgw_status fail(dgw_status s, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
static dgw_status fail(dgw_status s, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

#define DGW_CUDA(call)                                                                    \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(DGW_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                        __FILE__, __LINE__);                                              \
    } while (0)

using GraphKey = std::tuple<void*, double, int, cudaStream_t>;
// (U_in, U_out, dt, stream, copy flags) of a pipelined host step
using BandKey = std::tuple<const void*, void*, double, cudaStream_t, int>;

struct dgw_ctx {
    int device = 0;
    dgw_mesh mesh{};
    int p = 0;
    dgw_flux flux{};
    dgw_params params{};
    int K = 0;
    int64_t E = 0;
    int eb = 8;
    double h = 0.0;
    void* S1 = nullptr;
    void* S2 = nullptr;
    void* Uhost_dev = nullptr;   // device copy for dgw_rk_step_host
    double* partial = nullptr;   // mass partial sums
    double* mass_dev = nullptr;
    unsigned* flag = nullptr;
    double* t_dev = nullptr;     // the context's time (DGW_BC_STATE sides), advanced per step
    bool state_sides = false;
    int wait_limit = 0;          // bounded TMA waits: 0 the kernels' default limit (dgw_debug)
    int stage_kernel = 0;        // dgw_set_stage_kernel
    std::map<GraphKey, cudaGraphExec_t> graphs;
    std::map<std::pair<const void*, int>, CUtensorMap> tmaps;   // TMA descriptors (2D): (array, box kind)
    void* adj_ws = nullptr;      // adjoint: per-cell partials (own), K*E
    void* adj_wn = nullptr;      // adjoint: per-cell partials (one block per face), 2*dim*K*E
    void* adj_b1 = nullptr;      // adjoint: lambda of stage 2
    void* adj_b2 = nullptr;      // adjoint: lambda of stage 1
    std::map<std::pair<const void*, int>, bool> no_tmap;
    // dgw_rk_step_host pipeline: streams for input copies, output copies and a pool per
    // stage; one event per (input copy or stage, band); the join events
    cudaStream_t band_st[2 + 3 * 4] = {};
    cudaEvent_t band_ev[4][16] = {};
    cudaEvent_t band_join[2] = {};
    std::map<BandKey, cudaGraphExec_t> band_graphs;   // null: replay not possible (direct launches)
};

static const int kBands = 16;
static const int kStageStreams = 4;          // band kernels of one stage run concurrently
static const int kBandStreams = 2 + 3 * kStageStreams;

static const int kMassBlocks = 1024;
static const int kMassThreads = 256;

extern "C" void dgw_defaults(dgw_mesh* m, dgw_flux* f, dgw_params* s)
{
    if (m) {
        std::memset(m, 0, sizeof *m);
        m->dim = 1; m->nx = 16; m->ny = 1;
        m->x0 = 0.0; m->x1 = 1.0; m->y0 = 0.0; m->y1 = 1.0;
        for (int i = 0; i < 4; ++i) m->bc[i] = DGW_BC_PERIODIC;
    }
    if (f) {
        std::memset(f, 0, sizeof *f);
        f->kind = DGW_FLUX_ADVECT; f->a[0] = 1.0; f->a[1] = 0.0;
        f->center[0] = f->center[1] = 0.5; f->omega = 1.0; f->lambda_nu = 0.0; f->gas_gamma = 1.4;
    }
    if (s) {
        std::memset(s, 0, sizeof *s);
        s->stab = DGW_STAB_WENO; s->q = 1.0; s->b = 0.1; s->w_nbr = 1e-2;
        s->eps_w = 1e-6; s->eps_s = 1e-12; s->prec = DGW_FP64; s->theta = 1.0; s->rk_order = 3;
    }
}

static dgw_status check_params(const dgw_params* s, int dim)
{
    if (!s) return fail(DGW_EINVAL, "params is NULL");
    if (s->stab < DGW_STAB_DG || s->stab > DGW_STAB_ZHAO) return fail(DGW_EINVAL, "bad stab %d", s->stab);
    if (s->prec != DGW_FP64 && s->prec != DGW_FP32) return fail(DGW_EINVAL, "bad prec %d", s->prec);
    if (!(s->q > 0.0) || !std::isfinite(s->q)) return fail(DGW_EINVAL, "q must be > 0");
    if (!(s->b >= 0.0 && s->b <= 1.0)) return fail(DGW_EINVAL, "b must lie in [0, 1]");
    if (!(s->w_nbr >= 0.0 && s->w_nbr * 2 * dim < 1.0))
        return fail(DGW_EINVAL, "w_nbr must lie in [0, 1/(2 dim))");
    if (!(s->eps_w > 0.0) || !(s->eps_s >= 0.0)) return fail(DGW_EINVAL, "eps_w > 0 and eps_s >= 0 required");
    if (s->stab == DGW_STAB_ZHAO && !(s->w_nbr > 0.0 && s->theta > 0.0 && std::isfinite(s->theta)))
        return fail(DGW_EINVAL, "the ZHAO sensor needs w_nbr > 0 and a finite theta > 0");
    if (s->rk_order < 2 || s->rk_order > 4) return fail(DGW_EINVAL, "rk_order must be 2, 3 or 4");
    return DGW_OK;
}

extern "C" dgw_status dgw_create(const dgw_mesh* mesh, int p, const dgw_flux* flux,
                                 const dgw_params* params, dgw_ctx** out)
{
    if (!mesh || !flux || !params || !out) return fail(DGW_EINVAL, "NULL argument to dgw_create");
    *out = nullptr;
    const dgw_mesh& m = *mesh;
    if (m.dim != 1 && m.dim != 2) return fail(DGW_EINVAL, "dim must be 1 or 2");
    if (m.nx < 1 || (m.dim == 2 && m.ny < 1)) return fail(DGW_EINVAL, "nx, ny must be >= 1");
    if (!(m.x1 > m.x0) || (m.dim == 2 && !(m.y1 > m.y0))) return fail(DGW_EINVAL, "empty box");
    for (int f = 0; f < 2 * m.dim; ++f)
        if (m.bc[f] < DGW_BC_PERIODIC || m.bc[f] > DGW_BC_STATE) return fail(DGW_EINVAL, "bad bc[%d]", f);
    for (int a = 0; a < m.dim; ++a)
        if ((m.bc[2 * a] == DGW_BC_PERIODIC) != (m.bc[2 * a + 1] == DGW_BC_PERIODIC))
            return fail(DGW_EINVAL, "periodic sides must come in pairs");
    const double hx = (m.x1 - m.x0) / m.nx;
    if (m.dim == 2) {
        const double hy = (m.y1 - m.y0) / m.ny;
        if (std::fabs(hx - hy) > 1e-12 * hx) return fail(DGW_EUNSUPPORTED, "2D cells must be square");
    }
    if (p < 1 || p > kMaxP) return fail(DGW_EUNSUPPORTED, "degree p=%d not built (1..3)", p);
    if (flux->kind < DGW_FLUX_ADVECT || flux->kind > DGW_FLUX_EULER) return fail(DGW_EINVAL, "bad flux kind");
    if (!(flux->lambda_nu >= 0.0)) return fail(DGW_EINVAL, "lambda_nu must be >= 0");
    const bool euler = flux->kind == DGW_FLUX_EULER;
    bool state_sides = false;
    for (int f = 0; f < 2 * m.dim; ++f) {
        if (m.bc[f] == DGW_BC_REFLECT && !euler) return fail(DGW_EINVAL, "bc[%d]: reflecting walls are for the Euler system", f);
        if (m.bc[f] == DGW_BC_INFLOW_ZERO && euler) return fail(DGW_EINVAL, "bc[%d]: inflow_zero is for scalar laws", f);
        if (m.bc[f] == DGW_BC_STATE) {
            if (!euler || m.dim != 2) return fail(DGW_EUNSUPPORTED, "bc[%d]: prescribed states are built for the 2D Euler system", f);
            if (flux->bbelow[f] < 0 || flux->bbelow[f] > 2 || flux->babove[f] < 0 || flux->babove[f] > 2)
                return fail(DGW_EINVAL, "bc[%d]: bbelow / babove must be 0, 1 (a state) or 2 (a wall)", f);
            if (!std::isfinite(flux->bsplit[f]) || !std::isfinite(flux->bspeed[f]))
                return fail(DGW_EINVAL, "bc[%d]: bsplit and bspeed must be finite", f);
            state_sides = true;
        }
    }
    if (state_sides && params->rk_order == 4)
        return fail(DGW_EUNSUPPORTED, "prescribed states with rk_order 4: the stage times are built for orders 2 and 3");
    if (euler && !(flux->gas_gamma > 1.0 && std::isfinite(flux->gas_gamma)))
        return fail(DGW_EINVAL, "gas_gamma must be a finite number > 1");
    dgw_status st = check_params(params, m.dim);
    if (st != DGW_OK) return st;
    const int64_t E = m.dim == 1 ? (int64_t)m.nx : (int64_t)m.nx * m.ny;
    if (E > ((int64_t)1 << 36)) return fail(DGW_EINVAL, "mesh too large");

    dgw_ctx* c = new dgw_ctx();
    c->mesh = m;
    if (m.dim == 1) { c->mesh.ny = 1; }
    c->p = p;
    c->flux = *flux;
    c->params = *params;
    c->K = (m.dim == 1 ? p + 1 : (p + 1) * (p + 1)) * (euler ? m.dim + 2 : 1);
    c->E = E;
    c->eb = params->prec == DGW_FP64 ? 8 : 4;
    c->h = hx;
    cudaError_t ce = cudaGetDevice(&c->device);
    HostTables t;
    build_tables(p, &t);
    if (ce == cudaSuccess) {
        if (params->prec == DGW_FP64) ce = m.dim == 1 ? upload_tables_f64_d1(t) : upload_tables_f64_d2(t);
        else ce = m.dim == 1 ? upload_tables_f32_d1(t) : upload_tables_f32_d2(t);
    }
    const size_t bytes = (size_t)c->K * E * c->eb;
    if (ce == cudaSuccess) ce = cudaMalloc(&c->S1, bytes);
    if (ce == cudaSuccess) ce = cudaMalloc(&c->S2, bytes);
    if (ce == cudaSuccess) ce = cudaMalloc(&c->partial, sizeof(double) * (kMassBlocks + 2));
    if (ce == cudaSuccess) ce = cudaMemset(c->partial + kMassBlocks + 1, 0, sizeof(double));   // t = 0
    if (ce == cudaSuccess) ce = cudaMalloc(&c->flag, sizeof(unsigned));
    if (ce == cudaSuccess) ce = cudaMemset(c->flag, 0, sizeof(unsigned));
    if (ce != cudaSuccess) {
        dgw_status s = fail(ce == cudaErrorMemoryAllocation ? DGW_ENOMEM : DGW_ECUDA,
                            "dgw_create: %s", cudaGetErrorString(ce));
        dgw_destroy(c);
        return s;
    }
    c->mass_dev = c->partial + kMassBlocks;
    c->t_dev = c->partial + kMassBlocks + 1;
    c->state_sides = state_sides;
    *out = c;
    return DGW_OK;
}

static void drop_graphs(dgw_ctx* c)
{
    for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second);
    c->graphs.clear();
    for (auto& kv : c->band_graphs)
        if (kv.second) cudaGraphExecDestroy(kv.second);
    c->band_graphs.clear();
}

extern "C" dgw_status dgw_destroy(dgw_ctx* c)
{
    if (!c) return DGW_OK;
    cudaDeviceSynchronize();
    drop_graphs(c);
    cudaFree(c->S1);
    cudaFree(c->S2);
    cudaFree(c->Uhost_dev);
    cudaFree(c->adj_ws);
    cudaFree(c->adj_wn);
    cudaFree(c->adj_b1);
    cudaFree(c->adj_b2);
    cudaFree(c->partial);
    cudaFree(c->flag);
    for (int i = 0; i < kBandStreams; ++i)
        if (c->band_st[i]) cudaStreamDestroy(c->band_st[i]);
    for (int i = 0; i < 4; ++i)
        for (int b = 0; b < kBands; ++b)
            if (c->band_ev[i][b]) cudaEventDestroy(c->band_ev[i][b]);
    for (int i = 0; i < 2; ++i)
        if (c->band_join[i]) cudaEventDestroy(c->band_join[i]);
    delete c;
    return DGW_OK;
}

extern "C" dgw_status dgw_sizes(const dgw_ctx* c, int64_t* E, int* K, int* eb)
{
    if (!c) return fail(DGW_EINVAL, "NULL context");
    if (E) *E = c->E;
    if (K) *K = c->K;
    if (eb) *eb = c->eb;
    return DGW_OK;
}

extern "C" dgw_status dgw_set_params(dgw_ctx* c, const dgw_params* s)
{
    if (!c) return fail(DGW_EINVAL, "NULL context");
    dgw_status st = check_params(s, c->mesh.dim);
    if (st != DGW_OK) return st;
    if (s->prec != c->params.prec) return fail(DGW_EINVAL, "precision is fixed at dgw_create");
    if (c->state_sides && s->rk_order == 4)
        return fail(DGW_EUNSUPPORTED, "prescribed states with rk_order 4: the stage times are built for orders 2 and 3");
    c->params = *s;
    drop_graphs(c);
    return DGW_OK;
}

// TMA descriptor of a state array viewed as a 3D tensor (x: nx, y: ny, k: K) with a
// stage-tile box.  Null when TMA does not apply: 1D meshes, or row / plane strides that
// are not multiples of 16 bytes.
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    static std::mutex mu;
    std::lock_guard<std::mutex> lock(mu);
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// box kind 0: tile plus halo (kBoxX2 x (rows + 2) x K); 1: tile (kTileX2 x rows x K),
// rows = stage_rows() of the context's precision; kinds 2 and 3: the same with rows =
// kPRows (the persistent float kernel).  True and the descriptor in *out if TMA applies.  The descriptor is copied out: the cache evicts all its entries when it grows
// past 64 arrays, so a pointer into it would not outlive the next lookup.
static bool tensor_map(const dgw_ctx* cc, const void* U, int kind, CUtensorMap* out)
{
    dgw_ctx* c = const_cast<dgw_ctx*>(cc);
    if (c->mesh.dim != 2 || !U || c->flux.kind == DGW_FLUX_EULER) return false;   // the Euler kernel stages by plain loads
    const auto key = std::make_pair(U, kind);
    auto it = c->tmaps.find(key);
    if (it != c->tmaps.end()) {
        *out = it->second;
        return true;
    }
    if (c->no_tmap.count(key)) return false;
    if (c->tmaps.size() + c->no_tmap.size() > 64) {
        c->tmaps.clear();
        c->no_tmap.clear();
    }
    const uint64_t eb = (uint64_t)c->eb, nx = (uint64_t)c->mesh.nx, ny = (uint64_t)c->mesh.ny;
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc || (nx * eb) % 16 || (nx * ny * eb) % 16 || ((uintptr_t)U & 15u)) {
        c->no_tmap[key] = true;
        return false;
    }
    cuuint64_t dims[3] = {nx, ny, (cuuint64_t)c->K};
    cuuint64_t strides[2] = {nx * eb, nx * ny * eb};
    const int rows = kind >= 2 ? kPRows : stage_rows(eb == 8);
    const bool halo = kind == 0 || kind == 2;
    cuuint32_t box[3] = {(cuuint32_t)(halo ? kBoxX2 : kTileX2), (cuuint32_t)(halo ? rows + 2 : rows),
                         (cuuint32_t)c->K};
    cuuint32_t estr[3] = {1, 1, 1};
    CUtensorMap m;
    CUresult r = enc(&m, eb == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                     const_cast<void*>(U), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        c->no_tmap[key] = true;
        return false;
    }
    c->tmaps[key] = m;
    *out = m;
    return true;
}

static StageArgs base_args(const dgw_ctx* c)
{
    StageArgs a;
    std::memset(&a, 0, sizeof a);
    a.E = c->E;
    a.nx = c->mesh.nx;
    a.ny = c->mesh.dim == 2 ? c->mesh.ny : 1;
    a.x0 = c->mesh.x0;
    a.y0 = c->mesh.y0;
    a.h = c->h;
    for (int f = 0; f < 4; ++f) a.bc[f] = c->mesh.bc[f];
    a.a0 = c->flux.a[0];
    a.a1 = c->flux.a[1];
    a.cx = c->flux.center[0];
    a.cy = c->flux.center[1];
    a.omega = c->flux.omega;
    a.lambda_nu = c->flux.lambda_nu;
    a.stab = c->params.stab;
    a.q = c->params.q;
    a.b = c->params.b;
    a.w_nbr = c->params.w_nbr;
    a.eps_w = c->params.eps_w;
    a.eps_s = c->params.eps_s;
    a.theta = c->params.theta;
    a.gas_gamma = c->flux.gas_gamma;
    a.flag = c->flag;
    a.wait_limit = c->wait_limit;
    a.kernel_choice = c->stage_kernel;
    a.t_dev = c->t_dev;
    a.t_off = 0.0;
    for (int i = 0; i < 2; ++i)
        for (int k = 0; k < 4; ++k) a.bstate[i][k] = c->flux.bstate[i][k];
    for (int f = 0; f < 4; ++f) {
        a.bsplit[f] = c->flux.bsplit[f];
        a.bspeed[f] = c->flux.bspeed[f];
        a.bbelow[f] = c->flux.bbelow[f];
        a.babove[f] = c->flux.babove[f];
    }
    return a;
}

// t += dt on the device, after each step of a context with prescribed-state sides
__global__ void advance_time_kernel(double* t, double dt) { *t += dt; }

static cudaError_t launch(const dgw_ctx* c, const StageArgs& a0, int mode, cudaStream_t s)
{
    StageArgs a = a0;
    CUtensorMap m_k, m_n, m_pk, m_pn;      // copies: the launch parameters take them by value
    a.tmap = tensor_map(c, a.Uk, 0, &m_k) ? &m_k : nullptr;
    a.tmap_un = (a.cn != 0.0 && a.Un && tensor_map(c, a.Un, 1, &m_n)) ? &m_n : nullptr;
    const bool f64 = c->params.prec == DGW_FP64;
    a.tmap_p = a.tmap_un_p = nullptr;
    // whole-mesh float stage launches run the persistent kernel when its boxes apply
    // (the Un box too, where the stage reads Un)
    if (!f64 && c->mesh.dim == 2 && mode == 0 && a.kernel_choice != 1 && a.tile_row0 == 0 && a.tile_rows == 0 &&
        a.tmap && tensor_map(c, a.Uk, 2, &m_pk)) {
        const bool need_un = a.cn != 0.0 && a.Un;
        if (!need_un || (a.tmap_un && tensor_map(c, a.Un, 3, &m_pn))) {
            a.tmap_p = &m_pk;
            a.tmap_un_p = need_un ? &m_pn : nullptr;
        }
    }
    if (c->mesh.dim == 1)
        return f64 ? launch_stage_f64_d1(a, c->p, c->flux.kind, mode, s)
                   : launch_stage_f32_d1(a, c->p, c->flux.kind, mode, s);
    return f64 ? launch_stage_f64_d2(a, c->p, c->flux.kind, mode, s)
               : launch_stage_f32_d2(a, c->p, c->flux.kind, mode, s);
}

static bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

static dgw_status check_ctx(const dgw_ctx* c)
{
    if (!c) return fail(DGW_EINVAL, "NULL context");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != c->device)
        return fail(DGW_EINVAL, "context belongs to device %d, current device is %d", c->device, dev);
    return DGW_OK;
}

extern "C" dgw_status dgw_residual(dgw_ctx* c, const void* U, void* L, void* stream)
{
    dgw_status st = check_ctx(c);
    if (st != DGW_OK) return st;
    if (!U || !L) return fail(DGW_EINVAL, "NULL array");
    if (!aligned16(U) || !aligned16(L)) return fail(DGW_EINVAL, "arrays must be 16-byte aligned");
    if (U == L) return fail(DGW_EINVAL, "U and L must not overlap");
    StageArgs a = base_args(c);
    a.Uk = U;
    a.Uout = L;
    a.cn = 0.0; a.ck = 0.0; a.cl = 1.0;
    DGW_CUDA(launch(c, a, 0, (cudaStream_t)stream));
    return DGW_OK;
}

extern "C" dgw_status dgw_sensor(dgw_ctx* c, const void* U, double* gamma, void* stream)
{
    dgw_status st = check_ctx(c);
    if (st != DGW_OK) return st;
    if (!U || !gamma) return fail(DGW_EINVAL, "NULL array");
    if (!aligned16(U)) return fail(DGW_EINVAL, "U must be 16-byte aligned");
    StageArgs a = base_args(c);
    a.Uk = U;
    a.gamma_out = gamma;
    DGW_CUDA(launch(c, a, 1, (cudaStream_t)stream));
    return DGW_OK;
}

// The register recombination of the ten-stage SSP method of order 4:
// q2 <- q2/25 + 9/25 q1, then q1 <- 15 q2 - 5 q1 (with the new q2).
template <typename Real>
__global__ void rk4_mix_kernel(Real* __restrict__ q2, Real* __restrict__ q1, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const Real b = q2[i] / Real(25) + Real(9) / Real(25) * q1[i];
        q2[i] = b;
        q1[i] = Real(15) * b - Real(5) * q1[i];
    }
}

// SSP Runge-Kutta of order 2 and 4 (c->params.rk_order; Sec. 5 integrates with order
// p + 1).  Order 2: S1 = U + dt L(U); U <- 1/2 U + 1/2 (S1 + dt L(S1)).  Order 4 (the
// ten-stage method of Ketcheson): q2 lives in U, q1 alternates between S1 and S2;
// five stages q1 <- q1 + dt/6 L(q1), the recombination, four more, and
// U <- q2 + 3/5 q1 + dt/10 L(q1).  Final stages write U in place (own-element reads).
static cudaError_t enqueue_steps_rk24(const dgw_ctx* c, void* U, double dt, int nsteps, cudaStream_t s)
{
    StageArgs a = base_args(c);
    for (int n = 0; n < nsteps; ++n) {
        if (c->params.rk_order == 2) {
            a.Uk = U; a.Un = nullptr; a.Uout = c->S1;
            a.cn = 0.0; a.ck = 1.0; a.cl = dt; a.t_off = 0.0;
            cudaError_t e = launch(c, a, 0, s);
            if (e != cudaSuccess) return e;
            a.Uk = c->S1; a.Un = U; a.Uout = U;
            a.cn = 0.5; a.ck = 0.5; a.cl = 0.5 * dt; a.t_off = dt;
            e = launch(c, a, 0, s);
            if (e != cudaSuccess) return e;
            if (c->state_sides) {
                advance_time_kernel<<<1, 1, 0, s>>>(c->t_dev, dt);
                e = cudaGetLastError();
                if (e != cudaSuccess) return e;
            }
            continue;
        }
        void* q[2] = {c->S1, c->S2};
        int cur = 0;                       // q1 is q[cur]
        a.Un = nullptr; a.cn = 0.0; a.ck = 1.0; a.cl = dt / 6.0;
        for (int k = 0; k < 9; ++k) {
            a.Uk = k == 0 ? U : q[cur];
            a.Uout = k == 0 ? q[0] : q[cur ^ 1];
            cudaError_t e = launch(c, a, 0, s);
            if (e != cudaSuccess) return e;
            if (k > 0) cur ^= 1;
            if (k == 4) {
                const int64_t N = (int64_t)c->K * c->E;
                const unsigned blocks = (unsigned)std::min<int64_t>((N + 255) / 256, 152 * 16);
                if (c->eb == 8) rk4_mix_kernel<double><<<blocks, 256, 0, s>>>((double*)U, (double*)q[cur], N);
                else rk4_mix_kernel<float><<<blocks, 256, 0, s>>>((float*)U, (float*)q[cur], N);
                e = cudaGetLastError();
                if (e != cudaSuccess) return e;
            }
        }
        a.Uk = q[cur]; a.Un = U; a.Uout = U;
        a.cn = 1.0; a.ck = 3.0 / 5.0; a.cl = dt / 10.0;
        cudaError_t e = launch(c, a, 0, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// One SSP-RK3 step (Eq. ssp): U1 = U + dt L(U); U2 = 3/4 U + 1/4 (U1 + dt L(U1));
// U <- 1/3 U + 2/3 (U2 + dt L(U2)).  The third stage writes U in place: each thread
// reads U only at its own element there.  Other orders: enqueue_steps_rk24.
static cudaError_t enqueue_steps(const dgw_ctx* c, void* U, double dt, int nsteps, cudaStream_t s)
{
    if (c->params.rk_order != 3) return enqueue_steps_rk24(c, U, dt, nsteps, s);
    StageArgs a = base_args(c);
    for (int n = 0; n < nsteps; ++n) {
        a.Uk = U; a.Un = nullptr; a.Uout = c->S1;
        a.cn = 0.0; a.ck = 1.0; a.cl = dt; a.t_off = 0.0;
        cudaError_t e = launch(c, a, 0, s);
        if (e != cudaSuccess) return e;
        a.Uk = c->S1; a.Un = U; a.Uout = c->S2;
        a.cn = 0.75; a.ck = 0.25; a.cl = 0.25 * dt; a.t_off = dt;
        e = launch(c, a, 0, s);
        if (e != cudaSuccess) return e;
        a.Uk = c->S2; a.Un = U; a.Uout = U;
        a.cn = 1.0 / 3.0; a.ck = 2.0 / 3.0; a.cl = 2.0 / 3.0 * dt; a.t_off = 0.5 * dt;
        e = launch(c, a, 0, s);
        if (e != cudaSuccess) return e;
        if (c->state_sides) {
            advance_time_kernel<<<1, 1, 0, s>>>(c->t_dev, dt);
            e = cudaGetLastError();
            if (e != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

static const int kGraphChunk = 16;

static dgw_status run_graph(dgw_ctx* c, void* U, double dt, int n, cudaStream_t s)
{
    GraphKey key{U, dt, n, s};
    auto it = c->graphs.find(key);
    cudaGraphExec_t exec = nullptr;
    if (it == c->graphs.end()) {
        if (c->graphs.size() >= 8) drop_graphs(c);
        cudaGraph_t g = nullptr;
        DGW_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = enqueue_steps(c, U, dt, n, s);
        cudaError_t e2 = cudaStreamEndCapture(s, &g);
        if (e != cudaSuccess || e2 != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return fail(DGW_ECUDA, "graph capture failed: %s",
                        cudaGetErrorString(e != cudaSuccess ? e : e2));
        }
        e = cudaGraphInstantiate(&exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return fail(DGW_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
        c->graphs[key] = exec;
    } else {
        exec = it->second;
    }
    DGW_CUDA(cudaGraphLaunch(exec, s));
    return DGW_OK;
}

extern "C" dgw_status dgw_rk_step(dgw_ctx* c, void* U, double dt, int nsteps, void* stream)
{
    dgw_status st = check_ctx(c);
    if (st != DGW_OK) return st;
    if (!U) return fail(DGW_EINVAL, "NULL state");
    if (!aligned16(U)) return fail(DGW_EINVAL, "U must be 16-byte aligned");
    if (nsteps < 0) return fail(DGW_EINVAL, "nsteps < 0");
    if (!std::isfinite(dt)) return fail(DGW_EINVAL, "dt must be finite");
    if (nsteps == 0) return DGW_OK;
    cudaStream_t s = (cudaStream_t)stream;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (s != nullptr) DGW_CUDA(cudaStreamIsCapturing(s, &cap));
    if (s == nullptr || cap != cudaStreamCaptureStatusNone) {
        DGW_CUDA(enqueue_steps(c, U, dt, nsteps, s));
        return DGW_OK;
    }
    const int full = nsteps / kGraphChunk, rest = nsteps % kGraphChunk;
    for (int i = 0; i < full; ++i) {
        st = run_graph(c, U, dt, kGraphChunk, s);
        if (st != DGW_OK) return st;
    }
    if (rest) return run_graph(c, U, dt, rest, s);
    return DGW_OK;
}

// One SSP-RK3 step of a 2D mesh that is not periodic in y, as a wavefront over bands of
// tile rows: stage r of band b reads stage r - 1 on bands b - 1 .. b + 1 only, and bands of
// one stage do not depend on each other.  So the input copy of a band, the three stages
// and the output copy of a finished band overlap, and band kernels of a stage run
// concurrently.  Streams: input copies (in order), output copies (in order), and a pool
// of kStageStreams per stage (band b on stream b mod kStageStreams); one event per (input
// copy or stage, band); all joined to the caller's stream s at both ends.  copy_in: U_in
// (host) is copied to c->Uhost_dev band by band first; copy_out: the result is copied to
// U_out band by band.  Stage 3 writes U in place; the old U of band b is still read by
// stage 1 of bands b - 1 and b + 1 (halo rows) and by stages 2, 3 of band b (own rows):
// stage 3 of band b waits for stage 2 of bands b - 1 .. b + 1, which waited for stage 1
// of bands b - 2 .. b + 2.
static dgw_status banded_step(dgw_ctx* c, const void* U_in, void* U_out, double dt, bool copy_in,
                              bool copy_out, cudaStream_t s)
{
    const int rows = stage_rows(c->eb == 8);
    const int trows = (c->mesh.ny + rows - 1) / rows;
    const int nb = trows < kBands ? trows : kBands;
    cudaStream_t* st = c->band_st;
    cudaStream_t in_st = st[0], out_st = st[1];
    auto stage_st = [&](int r, int b) { return st[2 + r * kStageStreams + b % kStageStreams]; };
    auto& ev = c->band_ev;
    DGW_CUDA(cudaEventRecord(c->band_join[0], s));
    for (int i = 0; i < kBandStreams; ++i) DGW_CUDA(cudaStreamWaitEvent(st[i], c->band_join[0], 0));

    int t0[kBands + 1];                 // band b: tile rows [t0[b], t0[b + 1])
    for (int b = 0; b <= nb; ++b) t0[b] = (int)((int64_t)trows * b / nb);
    const size_t eb = (size_t)c->eb, nx = (size_t)c->mesh.nx, pitch = (size_t)c->E * eb;
    auto row_span = [&](int b, size_t* off, size_t* width) {
        const int r0 = t0[b] * rows;
        const int r1 = t0[b + 1] * rows < c->mesh.ny ? t0[b + 1] * rows : c->mesh.ny;
        *off = (size_t)r0 * nx * eb;
        *width = (size_t)(r1 - r0) * nx * eb;
    };
    char* U = static_cast<char*>(c->Uhost_dev);
    if (copy_in)
        for (int b = 0; b < nb; ++b) {
            size_t off, width;
            row_span(b, &off, &width);
            DGW_CUDA(cudaMemcpy2DAsync(U + off, pitch, static_cast<const char*>(U_in) + off, pitch, width,
                                       (size_t)c->K, cudaMemcpyHostToDevice, in_st));
            DGW_CUDA(cudaEventRecord(ev[0][b], in_st));
        }
    StageArgs a = base_args(c);
    for (int r = 0; r < 3; ++r) {
        if (r == 0) { a.Uk = U; a.Un = nullptr; a.Uout = c->S1; a.cn = 0.0; a.ck = 1.0; a.cl = dt; }
        if (r == 1) { a.Uk = c->S1; a.Un = U; a.Uout = c->S2; a.cn = 0.75; a.ck = 0.25; a.cl = 0.25 * dt; }
        if (r == 2) { a.Uk = c->S2; a.Un = U; a.Uout = U; a.cn = 1.0 / 3.0; a.ck = 2.0 / 3.0; a.cl = 2.0 / 3.0 * dt; }
        for (int b = 0; b < nb; ++b) {
            cudaStream_t ks = stage_st(r, b);
            if (r == 0) {
                // the input copies complete in order: the highest band read suffices
                if (copy_in) DGW_CUDA(cudaStreamWaitEvent(ks, ev[0][b + 1 < nb ? b + 1 : nb - 1], 0));
            } else {
                for (int d = b - 1; d <= b + 1; ++d)
                    if (d >= 0 && d < nb) DGW_CUDA(cudaStreamWaitEvent(ks, ev[r][d], 0));
            }
            a.tile_row0 = t0[b];
            a.tile_rows = t0[b + 1] - t0[b];
            DGW_CUDA(launch(c, a, 0, ks));
            DGW_CUDA(cudaEventRecord(ev[1 + r][b], ks));
        }
    }
    if (copy_out) {
        for (int b = 0; b < nb; ++b) {
            size_t off, width;
            row_span(b, &off, &width);
            DGW_CUDA(cudaStreamWaitEvent(out_st, ev[3][b], 0));
            DGW_CUDA(cudaMemcpy2DAsync(static_cast<char*>(U_out) + off, pitch, U + off, pitch, width,
                                       (size_t)c->K, cudaMemcpyDeviceToHost, out_st));
        }
        // the last output copy comes after every other operation (each copy waited for its
        // band's stage 3, which waited for everything before it)
        DGW_CUDA(cudaEventRecord(c->band_join[1], out_st));
        DGW_CUDA(cudaStreamWaitEvent(s, c->band_join[1], 0));
    } else {
        for (int b = 0; b < nb; ++b) DGW_CUDA(cudaStreamWaitEvent(s, ev[3][b], 0));
    }
    return DGW_OK;
}

static dgw_status band_resources(dgw_ctx* c)
{
    for (int i = 0; i < kBandStreams; ++i)
        if (!c->band_st[i]) DGW_CUDA(cudaStreamCreateWithFlags(&c->band_st[i], cudaStreamNonBlocking));
    for (int i = 0; i < 4; ++i)
        for (int b = 0; b < kBands; ++b)
            if (!c->band_ev[i][b]) DGW_CUDA(cudaEventCreateWithFlags(&c->band_ev[i][b], cudaEventDisableTiming));
    for (int i = 0; i < 2; ++i)
        if (!c->band_join[i]) DGW_CUDA(cudaEventCreateWithFlags(&c->band_join[i], cudaEventDisableTiming));
    return DGW_OK;
}

// banded_step, replayed from a graph cached per (U_in, U_out, dt, stream, copies) when the
// stream can be captured; launched directly otherwise (the legacy stream, a stream that is
// itself being captured, or host memory that a graph cannot copy from).
static dgw_status banded(dgw_ctx* c, const void* U_in, void* U_out, double dt, bool copy_in, bool copy_out,
                         cudaStream_t s)
{
    dgw_status st = band_resources(c);
    if (st != DGW_OK) return st;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (s != nullptr) DGW_CUDA(cudaStreamIsCapturing(s, &cap));
    if (s == nullptr || cap != cudaStreamCaptureStatusNone) return banded_step(c, U_in, U_out, dt, copy_in, copy_out, s);
    const BandKey key{U_in, U_out, dt, s, (copy_in ? 1 : 0) | (copy_out ? 2 : 0)};
    auto it = c->band_graphs.find(key);
    if (it == c->band_graphs.end()) {
        if (c->band_graphs.size() >= 8) {
            for (auto& kv : c->band_graphs)
                if (kv.second) cudaGraphExecDestroy(kv.second);
            c->band_graphs.clear();
        }
        cudaGraphExec_t exec = nullptr;
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            const dgw_status sc = banded_step(c, U_in, U_out, dt, copy_in, copy_out, s);
            const cudaError_t e = cudaStreamEndCapture(s, &g);
            if (sc == DGW_OK && e == cudaSuccess && g && cudaGraphInstantiate(&exec, g, 0) != cudaSuccess) exec = nullptr;
            if (g) cudaGraphDestroy(g);
        }
        cudaGetLastError();    // a refused capture leaves no error behind for later calls
        it = c->band_graphs.emplace(key, exec).first;
    }
    if (!it->second) return banded_step(c, U_in, U_out, dt, copy_in, copy_out, s);
    DGW_CUDA(cudaGraphLaunch(it->second, s));
    return DGW_OK;
}

extern "C" dgw_status dgw_rk_step_host(dgw_ctx* c, const void* U_in, void* U_out, double dt,
                                       int nsteps, void* stream)
{
    dgw_status st = check_ctx(c);
    if (st != DGW_OK) return st;
    if (!U_in || !U_out) return fail(DGW_EINVAL, "NULL host array");
    if (nsteps < 1) return fail(DGW_EINVAL, "nsteps < 1");
    if (!std::isfinite(dt)) return fail(DGW_EINVAL, "dt must be finite");
    const size_t bytes = (size_t)c->K * c->E * c->eb;
    if (!c->Uhost_dev) {
        cudaError_t e = cudaMalloc(&c->Uhost_dev, bytes);
        if (e != cudaSuccess) return fail(DGW_ENOMEM, "dgw_rk_step_host: %s", cudaGetErrorString(e));
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int rows = stage_rows(c->eb == 8);
    const bool pipelined = c->mesh.dim == 2 && c->mesh.bc[2] != DGW_BC_PERIODIC && c->mesh.ny >= 2 * rows &&
                           c->params.rk_order == 3 && c->flux.kind != DGW_FLUX_EULER;
    if (!pipelined) {
        DGW_CUDA(cudaMemcpyAsync(c->Uhost_dev, U_in, bytes, cudaMemcpyHostToDevice, s));
        st = dgw_rk_step(c, c->Uhost_dev, dt, nsteps, stream);
        if (st != DGW_OK) return st;
        DGW_CUDA(cudaMemcpyAsync(U_out, c->Uhost_dev, bytes, cudaMemcpyDeviceToHost, s));
    } else if (nsteps == 1) {
        st = banded(c, U_in, U_out, dt, true, true, s);
        if (st != DGW_OK) return st;
    } else {
        st = banded(c, U_in, nullptr, dt, true, false, s);
        if (st == DGW_OK && nsteps > 2) st = dgw_rk_step(c, c->Uhost_dev, dt, nsteps - 2, stream);
        if (st == DGW_OK) st = banded(c, nullptr, U_out, dt, false, true, s);
        if (st != DGW_OK) return st;
    }
    DGW_CUDA(cudaStreamSynchronize(s));
    return DGW_OK;
}

// ------------------------------------------------------------------------------------
// projection
// ------------------------------------------------------------------------------------
struct ProjArgs {
    const double* f;
    void* U;
    int64_t E;
    int nq, n1, dim, f64;
    double w[8];
    double B[8][kMaxN1];
    double minv[kMaxN1];
};

__global__ void project_kernel(const ProjArgs a)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= a.E) return;
    const int npt = a.dim == 1 ? a.nq : a.nq * a.nq;
    const double* f = a.f + e * npt;
    const int K = a.dim == 1 ? a.n1 : a.n1 * a.n1;
    for (int k = 0; k < K; ++k) {
        const int i = k % a.n1, j = k / a.n1;
        double s = 0.0;
        if (a.dim == 1) {
            for (int q = 0; q < a.nq; ++q) s += a.w[q] * a.B[q][i] * f[q];
            s *= a.minv[i];
        } else {
            for (int qb = 0; qb < a.nq; ++qb) {
                double r = 0.0;
                for (int qa = 0; qa < a.nq; ++qa) r += a.w[qa] * a.B[qa][i] * f[qa + a.nq * qb];
                s += a.w[qb] * a.B[qb][j] * r;
            }
            s *= a.minv[i] * a.minv[j];
        }
        if (a.f64) static_cast<double*>(a.U)[k * a.E + e] = s;
        else static_cast<float*>(a.U)[k * a.E + e] = (float)s;
    }
}


extern "C" dgw_status dgw_project(dgw_ctx* c, int nq, const double* samples, void* U, void* stream)
{
    dgw_status st = check_ctx(c);
    if (st != DGW_OK) return st;
    if (!samples || !U) return fail(DGW_EINVAL, "NULL array");
    if (nq < 1 || nq > 8) return fail(DGW_EINVAL, "nq must lie in 1..8");
    ProjArgs a;
    std::memset(&a, 0, sizeof a);
    a.f = samples; a.U = U; a.E = c->E; a.nq = nq; a.n1 = c->p + 1; a.dim = c->mesh.dim;
    a.f64 = c->params.prec == DGW_FP64;
    double x[8];
    gauss_rule_public(nq, x, a.w);
    for (int q = 0; q < nq; ++q) {
        // P_0..P_p at x_q by the three-term recurrence
        double pm = 1.0, pc = x[q];
        a.B[q][0] = 1.0;
        if (c->p >= 1) a.B[q][1] = x[q];
        for (int k = 1; k < c->p; ++k) {
            double pn = ((2 * k + 1) * x[q] * pc - k * pm) / (k + 1);
            pm = pc; pc = pn;
            a.B[q][k + 1] = pn;
        }
    }
    for (int i = 0; i <= c->p; ++i) a.minv[i] = (2 * i + 1) / 2.0;
    const int threads = 128;
    const int64_t blocks = (c->E + threads - 1) / threads;
    // the Euler system: one projection per component (samples and rows component-major)
    const int ncomp = c->flux.kind == DGW_FLUX_EULER ? c->mesh.dim + 2 : 1;
    const int64_t npt = c->mesh.dim == 1 ? nq : nq * nq;
    for (int comp = 0; comp < ncomp; ++comp) {
        a.f = samples + comp * c->E * npt;
        a.U = static_cast<char*>(U) + (size_t)comp * (c->K / ncomp) * c->E * c->eb;
        project_kernel<<<(unsigned)blocks, threads, 0, (cudaStream_t)stream>>>(a);
        DGW_CUDA(cudaGetLastError());
    }
    return DGW_OK;
}

// ------------------------------------------------------------------------------------
// batched ensemble
// ------------------------------------------------------------------------------------
struct dgw_batch {
    int device = 0;
    int n = 0;
    dgw_params params{};
    int eb = 4;
    std::vector<BatchInst> inst;
    std::vector<int> dims;
    int64_t total = 0;
    BatchInst* d_inst = nullptr;
    // per group (dimension, degree): its work items, kernel tile height, items' chunk of
    // tiles, grid, and the stream its persistent kernel runs on
    BatchItem* d_items[2][kMaxP + 1] = {};
    int nitems[2][kMaxP + 1] = {};
    int rows[2][kMaxP + 1] = {};
    int chunk[2][kMaxP + 1] = {};
    int grid[2][kMaxP + 1] = {};
    void* S1 = nullptr;
    void* S2 = nullptr;
    unsigned long long* counters = nullptr;   // queue[kQueues], one per group, then done[n]
    unsigned* flag = nullptr;
    int* abort = nullptr;
    int sms = 0;
    long long wait_limit = 1ll << 24;
    int unreachable = 0;
    cudaStream_t st[2 * (kMaxP + 1)] = {};
    cudaEvent_t fork = nullptr;
    cudaEvent_t join[2 * (kMaxP + 1)] = {};
};

static const int kQueues = 2 * (kMaxP + 1);

static bool batch_group_used(const dgw_batch* b, int d, int p)
{
    for (int i = 0; i < b->n; ++i)
        if (b->dims[i] == d + 1 && b->inst[i].p == p) return true;
    return false;
}

static bool batch_rows_ok(const dgw_batch* b, int d, int rows)
{
    const bool f64 = b->eb == 8;
    return d == 0 ? (f64 ? batch_rows_built_f64_d1(rows) : batch_rows_built_f32_d1(rows))
                  : (f64 ? batch_rows_built_f64_d2(rows) : batch_rows_built_f32_d2(rows));
}

// Tiles of every instance of group (d, p) for the group's tile height, and the group's
// grid (resident CTAs per SM x SMs).  Uploads the instance table.
static dgw_status batch_layout(dgw_batch* b, int d, int p)
{
    const int rows = b->rows[d][p];
    for (int i = 0; i < b->n; ++i) {
        BatchInst& I = b->inst[i];
        if (b->dims[i] != d + 1 || I.p != p) continue;
        I.ntx = d == 0 ? (I.nx + 127) / 128 : (I.nx + kTileX2 - 1) / kTileX2;
        I.ntiles = d == 0 ? I.ntx : I.ntx * ((I.ny + rows - 1) / rows);
    }
    const bool f64 = b->eb == 8;
    const int bps = d == 0 ? (f64 ? batch_blocks_per_sm_f64_d1(p, rows) : batch_blocks_per_sm_f32_d1(p, rows))
                           : (f64 ? batch_blocks_per_sm_f64_d2(p, rows) : batch_blocks_per_sm_f32_d2(p, rows));
    if (bps <= 0) return fail(DGW_ECUDA, "batch kernel (dim %d, p %d, %d rows): occupancy query failed", d + 1, p, rows);
    b->grid[d][p] = bps * b->sms;
    DGW_CUDA(cudaMemcpy(b->d_inst, b->inst.data(), sizeof(BatchInst) * b->n, cudaMemcpyHostToDevice));
    return DGW_OK;
}

// Work items of group (d, p): chunks of the group's chunk size over each instance's
// tiles, longest instances first, so that the tail of each stage is made of small items.
static dgw_status batch_build_items(dgw_batch* b, int d, int p)
{
    std::vector<int> order;
    for (int i = 0; i < b->n; ++i)
        if (b->dims[i] == d + 1 && b->inst[i].p == p) order.push_back(i);
    std::stable_sort(order.begin(), order.end(),
                     [&](int x, int y) { return b->inst[x].ntiles > b->inst[y].ntiles; });
    const int c = b->chunk[d][p];
    std::vector<BatchItem> items;
    for (int i : order)
        for (int t = 0; t < b->inst[i].ntiles; t += c)
            items.push_back(BatchItem{i, t, std::min(c, b->inst[i].ntiles - t), 0});
    cudaFree(b->d_items[d][p]);
    b->d_items[d][p] = nullptr;
    b->nitems[d][p] = (int)items.size();
    if (!items.empty()) {
        DGW_CUDA(cudaMalloc(&b->d_items[d][p], sizeof(BatchItem) * items.size()));
        DGW_CUDA(cudaMemcpy(b->d_items[d][p], items.data(), sizeof(BatchItem) * items.size(),
                            cudaMemcpyHostToDevice));
    }
    return DGW_OK;
}

extern "C" dgw_status dgw_batch_destroy(dgw_batch* b)
{
    if (!b) return DGW_OK;
    cudaDeviceSynchronize();
    cudaFree(b->d_inst);
    for (int d = 0; d < 2; ++d)
        for (int p = 0; p <= kMaxP; ++p) cudaFree(b->d_items[d][p]);
    cudaFree(b->S1);
    cudaFree(b->S2);
    cudaFree(b->counters);
    cudaFree(b->flag);
    cudaFree(b->abort);
    for (int g = 0; g < 2 * (kMaxP + 1); ++g) {
        if (b->st[g]) cudaStreamDestroy(b->st[g]);
        if (b->join[g]) cudaEventDestroy(b->join[g]);
    }
    if (b->fork) cudaEventDestroy(b->fork);
    delete b;
    return DGW_OK;
}

extern "C" dgw_status dgw_batch_create(int n, const dgw_mesh* meshes, const int* ps, const dgw_flux* fluxes,
                                       const dgw_params* params, dgw_batch** out)
{
    if (!out || !meshes || !ps || !fluxes || !params || n < 1) return fail(DGW_EINVAL, "bad arguments to dgw_batch_create");
    *out = nullptr;
    dgw_status st = check_params(params, 2);
    if (params->rk_order != 3) return fail(DGW_EUNSUPPORTED, "the batch step is SSP-RK3 (rk_order 3)");
    if (st != DGW_OK) return st;
    std::vector<BatchInst> insts;
    std::vector<int> dims;
    int64_t off = 0;
    bool need_tab[2][2][kMaxP + 1] = {};
    const int eb = params->prec == DGW_FP64 ? 8 : 4;
    for (int i = 0; i < n; ++i) {
        const dgw_mesh& m = meshes[i];
        const int p = ps[i];
        const dgw_flux& f = fluxes[i];
        if (m.dim != 1 && m.dim != 2) return fail(DGW_EINVAL, "instance %d: dim must be 1 or 2", i);
        if (m.nx < 1 || (m.dim == 2 && m.ny < 1) || !(m.x1 > m.x0) || (m.dim == 2 && !(m.y1 > m.y0)))
            return fail(DGW_EINVAL, "instance %d: bad mesh", i);
        const double hx = (m.x1 - m.x0) / m.nx;
        if (m.dim == 2 && std::fabs(hx - (m.y1 - m.y0) / m.ny) > 1e-12 * hx)
            return fail(DGW_EUNSUPPORTED, "instance %d: 2D cells must be square", i);
        if (p < 1 || p > kMaxP) return fail(DGW_EUNSUPPORTED, "instance %d: degree %d not built", i, p);
        if (f.kind != DGW_FLUX_ADVECT && f.kind != DGW_FLUX_BURGERS)
            return fail(DGW_EUNSUPPORTED, "instance %d: the batched kernel is built for advection and Burgers", i);
        if (!(f.lambda_nu >= 0.0)) return fail(DGW_EINVAL, "instance %d: lambda_nu must be >= 0", i);
        for (int s = 0; s < 2 * m.dim; ++s)
            if (m.bc[s] < DGW_BC_PERIODIC || m.bc[s] > DGW_BC_OUTFLOW) return fail(DGW_EINVAL, "instance %d: bad bc", i);
        for (int a = 0; a < m.dim; ++a)
            if ((m.bc[2 * a] == DGW_BC_PERIODIC) != (m.bc[2 * a + 1] == DGW_BC_PERIODIC))
                return fail(DGW_EINVAL, "instance %d: periodic sides must come in pairs", i);
        BatchInst I;
        std::memset(&I, 0, sizeof I);
        I.nx = m.nx;
        I.ny = m.dim == 2 ? m.ny : 1;
        I.E = (int64_t)I.nx * I.ny;
        I.p = p;
        I.flux = f.kind;
        const int K = m.dim == 1 ? p + 1 : (p + 1) * (p + 1);
        for (int s = 0; s < 4; ++s) I.bc[s] = s < 2 * m.dim ? m.bc[s] : DGW_BC_PERIODIC;
        I.x0 = m.x0; I.y0 = m.y0; I.h = hx;
        I.a0 = f.a[0]; I.a1 = f.a[1]; I.cx = f.center[0]; I.cy = f.center[1];
        I.omega = f.omega; I.lambda_nu = f.lambda_nu; I.dt = 0.0;
        I.off = off;
        off += ((int64_t)K * I.E + 3) / 4 * 4;     // keep every instance 16-byte aligned
        insts.push_back(I);
        dims.push_back(m.dim);
        need_tab[eb == 8][m.dim - 1][p] = true;
    }
    dgw_batch* b = new dgw_batch();
    b->n = n;
    b->params = *params;
    b->eb = eb;
    b->inst = insts;
    b->dims = dims;
    b->total = off;
    cudaError_t ce = cudaGetDevice(&b->device);
    for (int f64 = 0; f64 < 2 && ce == cudaSuccess; ++f64)
        for (int d = 0; d < 2 && ce == cudaSuccess; ++d)
            for (int p = 1; p <= kMaxP && ce == cudaSuccess; ++p) {
                if (!need_tab[f64][d][p]) continue;
                HostTables t;
                build_tables(p, &t);
                ce = f64 ? (d == 0 ? upload_tables_f64_d1(t) : upload_tables_f64_d2(t))
                         : (d == 0 ? upload_tables_f32_d1(t) : upload_tables_f32_d2(t));
            }
    const size_t bytes = (size_t)b->total * b->eb;
    if (ce == cudaSuccess) ce = cudaMalloc(&b->S1, bytes);
    if (ce == cudaSuccess) ce = cudaMalloc(&b->S2, bytes);
    if (ce == cudaSuccess) ce = cudaMalloc(&b->counters, sizeof(unsigned long long) * (kQueues + n));
    if (ce == cudaSuccess) ce = cudaMalloc(&b->flag, sizeof(unsigned));
    if (ce == cudaSuccess) ce = cudaMemset(b->flag, 0, sizeof(unsigned));
    if (ce == cudaSuccess) ce = cudaMalloc(&b->abort, sizeof(int));
    if (ce == cudaSuccess) ce = cudaMalloc(&b->d_inst, sizeof(BatchInst) * n);
    if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device);
    if (ce != cudaSuccess) {
        dgw_status s2 = fail(ce == cudaErrorMemoryAllocation ? DGW_ENOMEM : DGW_ECUDA, "dgw_batch_create: %s",
                             cudaGetErrorString(ce));
        dgw_batch_destroy(b);
        return s2;
    }
    for (int g = 0; g < 2 * (kMaxP + 1) && ce == cudaSuccess; ++g) {
        ce = cudaStreamCreateWithFlags(&b->st[g], cudaStreamNonBlocking);
        if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&b->join[g], cudaEventDisableTiming);
    }
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    if (ce != cudaSuccess) {
        dgw_batch_destroy(b);
        return fail(DGW_ECUDA, "dgw_batch_create: %s", cudaGetErrorString(ce));
    }
    for (int d = 0; d < 2 && st == DGW_OK; ++d)
        for (int p = 1; p <= kMaxP && st == DGW_OK; ++p) {
            // default schedule (the autotuner's usual pick with pipelined staging): 1D
            // items of 2 tiles; 2D float tiles of 8 cell rows, items of 16 tiles
            const bool f64 = b->eb == 8;
            b->rows[d][p] = d == 0 ? 1 : (f64 ? kTileY2 : 8);
            b->chunk[d][p] = d == 0 ? 2 : 16;
            if (!batch_group_used(b, d, p)) continue;
            st = batch_layout(b, d, p);
            if (st == DGW_OK) st = batch_build_items(b, d, p);
        }
    if (st != DGW_OK) {
        dgw_batch_destroy(b);
        return st;
    }
    *out = b;
    return DGW_OK;
}

extern "C" dgw_status dgw_batch_sizes(const dgw_batch* b, int64_t* total, int64_t* offsets)
{
    if (!b) return fail(DGW_EINVAL, "NULL batch");
    if (total) *total = b->total;
    if (offsets)
        for (int i = 0; i < b->n; ++i) offsets[i] = b->inst[i].off;
    return DGW_OK;
}

extern "C" dgw_status dgw_batch_set_dt(dgw_batch* b, const double* dt)
{
    if (!b || !dt) return fail(DGW_EINVAL, "NULL argument");
    for (int i = 0; i < b->n; ++i)
        if (!std::isfinite(dt[i]) || dt[i] == 0.0) return fail(DGW_EINVAL, "dt[%d] must be finite and nonzero", i);
    for (int i = 0; i < b->n; ++i) b->inst[i].dt = dt[i];
    DGW_CUDA(cudaMemcpy(b->d_inst, b->inst.data(), sizeof(BatchInst) * b->n, cudaMemcpyHostToDevice));
    return DGW_OK;
}

extern "C" dgw_status dgw_batch_project(dgw_batch* b, int nq, int first, int count, const double* samples,
                                        void* U, void* stream)
{
    if (!b || !samples || !U) return fail(DGW_EINVAL, "NULL argument");
    if (nq < 1 || nq > 8) return fail(DGW_EINVAL, "nq must lie in 1..8");
    if (first < 0 || count < 0 || first + count > b->n) return fail(DGW_EINVAL, "instance range out of bounds");
    double x[8], w[8];
    gauss_rule_public(nq, x, w);
    int64_t so = 0;
    for (int i = first; i < first + count; ++i) {
        const BatchInst& I = b->inst[i];
        ProjArgs a;
        std::memset(&a, 0, sizeof a);
        a.f = samples + so;
        so += I.E * (b->dims[i] == 1 ? nq : nq * nq);
        a.U = static_cast<char*>(U) + (size_t)I.off * b->eb;
        a.E = I.E; a.nq = nq; a.n1 = I.p + 1; a.dim = b->dims[i]; a.f64 = b->eb == 8;
        for (int q = 0; q < nq; ++q) {
            a.w[q] = w[q];
            double pm = 1.0, pc = x[q];
            a.B[q][0] = 1.0;
            a.B[q][1] = x[q];
            for (int k = 1; k < I.p; ++k) {
                double pn = ((2 * k + 1) * x[q] * pc - k * pm) / (k + 1);
                pm = pc; pc = pn;
                a.B[q][k + 1] = pn;
            }
        }
        for (int k = 0; k <= I.p; ++k) a.minv[k] = (2 * k + 1) / 2.0;
        project_kernel<<<(unsigned)((I.E + 127) / 128), 128, 0, (cudaStream_t)stream>>>(a);
        DGW_CUDA(cudaGetLastError());
    }
    return DGW_OK;
}

// Launch of group (d, p)'s persistent kernel on stream s: it advances the group's
// instances through all 3 * nsteps stages.
static dgw_status batch_launch_group(dgw_batch* b, int d, int p, void* U, int nsteps, cudaStream_t s)
{
    BatchArgs a;
    std::memset(&a, 0, sizeof a);
    a.inst = b->d_inst;
    a.items = b->d_items[d][p];
    a.nitems = b->nitems[d][p];
    a.nstages = 3 * nsteps;
    a.U = U;
    a.S1 = b->S1;
    a.S2 = b->S2;
    a.queue = b->counters + d * (kMaxP + 1) + p;
    a.done = b->counters + kQueues;
    a.flag = b->flag;
    a.abort = b->abort;
    a.stab = b->params.stab;
    a.q = b->params.q; a.b = b->params.b; a.w_nbr = b->params.w_nbr;
    a.eps_w = b->params.eps_w; a.eps_s = b->params.eps_s; a.theta = b->params.theta;
    a.wait_limit = b->wait_limit;
    a.unreachable = b->unreachable;
    const bool f64 = b->eb == 8;
    const int rows = b->rows[d][p], g = b->grid[d][p];
    cudaError_t e = d == 0 ? (f64 ? launch_batch_f64_d1(a, p, rows, g, s) : launch_batch_f32_d1(a, p, rows, g, s))
                           : (f64 ? launch_batch_f64_d2(a, p, rows, g, s) : launch_batch_f32_d2(a, p, rows, g, s));
    if (e != cudaSuccess) return fail(DGW_ECUDA, "batch launch: %s", cudaGetErrorString(e));
    return DGW_OK;
}

// The persistent kernels of all groups (or of group `only` = d * (kMaxP + 1) + p) side by
// side: each on the batch's stream of its group, forked from s after the counters are
// cleared and joined back into s.  Groups with more DOFs start first; the others fill the
// SMs as its CTAs drain.
static dgw_status batch_enqueue(dgw_batch* b, void* U, int nsteps, cudaStream_t s, int only = -1)
{
    DGW_CUDA(cudaMemsetAsync(b->counters, 0, sizeof(unsigned long long) * (kQueues + b->n), s));
    DGW_CUDA(cudaMemsetAsync(b->abort, 0, sizeof(int), s));
    std::vector<std::pair<double, int>> groups;
    for (int d = 0; d < 2; ++d)
        for (int p = 1; p <= kMaxP; ++p) {
            const int gi = d * (kMaxP + 1) + p;
            if (b->nitems[d][p] == 0 || (only >= 0 && gi != only)) continue;
            double dofs = 0.0;
            for (int i = 0; i < b->n; ++i)
                if (b->dims[i] == d + 1 && b->inst[i].p == p)
                    dofs += (double)b->inst[i].E * (d == 0 ? p + 1 : (p + 1) * (p + 1));
            groups.push_back({-dofs, gi});
        }
    std::sort(groups.begin(), groups.end());
    DGW_CUDA(cudaEventRecord(b->fork, s));
    for (const auto& gr : groups) {
        const int gi = gr.second, d = gi / (kMaxP + 1), p = gi % (kMaxP + 1);
        DGW_CUDA(cudaStreamWaitEvent(b->st[gi], b->fork, 0));
        dgw_status st = batch_launch_group(b, d, p, U, nsteps, b->st[gi]);
        if (st != DGW_OK) return st;
        DGW_CUDA(cudaEventRecord(b->join[gi], b->st[gi]));
        DGW_CUDA(cudaStreamWaitEvent(s, b->join[gi], 0));
    }
    return DGW_OK;
}

extern "C" dgw_status dgw_batch_rk_step(dgw_batch* b, void* U, int nsteps, void* stream)
{
    if (!b || !U) return fail(DGW_EINVAL, "NULL argument");
    if (nsteps < 0) return fail(DGW_EINVAL, "nsteps < 0");
    if (((uintptr_t)U & 15u) != 0) return fail(DGW_EINVAL, "U must be 16-byte aligned");
    if (nsteps == 0) return DGW_OK;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != b->device) return fail(DGW_EINVAL, "wrong device");
    for (int i = 0; i < b->n; ++i)
        if (b->inst[i].dt == 0.0) return fail(DGW_EINVAL, "dt not set (dgw_batch_set_dt)");
    return batch_enqueue(b, U, nsteps, (cudaStream_t)stream);
}

// For each group alone: time `steps` steps for every built tile height and every chunk of
// 1, 2, 4, 8, 16 tiles on a copy of U, and keep the fastest pair.
extern "C" dgw_status dgw_batch_autotune(dgw_batch* b, void* U, int steps, int* chosen_chunk, void* stream)
{
    if (!b || !U || steps < 1) return fail(DGW_EINVAL, "bad arguments");
    for (int i = 0; i < b->n; ++i)
        if (b->inst[i].dt == 0.0) return fail(DGW_EINVAL, "dt not set (dgw_batch_set_dt)");
    cudaStream_t s = (cudaStream_t)stream;
    void* tmp = nullptr;
    const size_t bytes = (size_t)b->total * b->eb;
    DGW_CUDA(cudaMalloc(&tmp, bytes));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int chunks[] = {1, 2, 4, 8, 16};
    const int heights[] = {1, 2, 4, 8};
    dgw_status st = DGW_OK;
    double best_dofs = -1.0;
    for (int d = 0; d < 2 && st == DGW_OK; ++d)
        for (int p = 1; p <= kMaxP && st == DGW_OK; ++p) {
            if (!batch_group_used(b, d, p)) continue;
            int best_rows = b->rows[d][p], best_chunk = b->chunk[d][p];
            float best_ms = 1e30f;
            for (int rows : heights) {
                if (!batch_rows_ok(b, d, rows)) continue;
                b->rows[d][p] = rows;
                st = batch_layout(b, d, p);
                for (int c : chunks) {
                    if (st != DGW_OK) break;
                    b->chunk[d][p] = c;
                    st = batch_build_items(b, d, p);
                    if (st != DGW_OK) break;
                    if (cudaMemcpyAsync(tmp, U, bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
                        st = fail(DGW_ECUDA, "copy");
                        break;
                    }
                    const int gi = d * (kMaxP + 1) + p;
                    st = batch_enqueue(b, tmp, 1, s, gi);    // warm-up
                    if (st != DGW_OK) break;
                    cudaEventRecord(e0, s);
                    st = batch_enqueue(b, tmp, steps, s, gi);
                    if (st != DGW_OK) break;
                    cudaEventRecord(e1, s);
                    cudaEventSynchronize(e1);
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    if (ms < best_ms) { best_ms = ms; best_rows = rows; best_chunk = c; }
                }
            }
            if (st != DGW_OK) break;
            b->rows[d][p] = best_rows;
            b->chunk[d][p] = best_chunk;
            st = batch_layout(b, d, p);
            if (st == DGW_OK) st = batch_build_items(b, d, p);
            double dofs = 0.0;
            for (int i = 0; i < b->n; ++i)
                if (b->dims[i] == d + 1 && b->inst[i].p == p) dofs += (double)b->inst[i].E;
            if (dofs > best_dofs && chosen_chunk) { best_dofs = dofs; *chosen_chunk = best_chunk; }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamSynchronize(s);
    cudaFree(tmp);
    return st;
}

extern "C" dgw_status dgw_batch_schedule(const dgw_batch* b, int dim, int p, int* rows, int* chunk)
{
    if (!b || (dim != 1 && dim != 2) || p < 1 || p > kMaxP) return fail(DGW_EINVAL, "bad arguments");
    if (rows) *rows = b->rows[dim - 1][p];
    if (chunk) *chunk = b->chunk[dim - 1][p];
    return DGW_OK;
}

extern "C" dgw_status dgw_batch_set_schedule(dgw_batch* b, int dim, int p, int rows, int chunk)
{
    if (!b || (dim != 1 && dim != 2) || p < 1 || p > kMaxP) return fail(DGW_EINVAL, "bad arguments");
    if (!batch_rows_ok(b, dim - 1, rows)) return fail(DGW_EINVAL, "tile height %d not built for dim %d", rows, dim);
    if (chunk < 1) return fail(DGW_EINVAL, "chunk must be >= 1");
    b->rows[dim - 1][p] = rows;
    b->chunk[dim - 1][p] = chunk;
    if (!batch_group_used(b, dim - 1, p)) return DGW_OK;
    dgw_status st = batch_layout(b, dim - 1, p);
    return st == DGW_OK ? batch_build_items(b, dim - 1, p) : st;
}

extern "C" dgw_status dgw_batch_sync_status(dgw_batch* b, void* stream)
{
    if (!b) return fail(DGW_EINVAL, "NULL batch");
    unsigned v = 0;
    cudaStream_t s = (cudaStream_t)stream;
    DGW_CUDA(cudaMemcpyAsync(&v, b->flag, sizeof v, cudaMemcpyDeviceToHost, s));
    DGW_CUDA(cudaMemsetAsync(b->flag, 0, sizeof(unsigned), s));
    DGW_CUDA(cudaStreamSynchronize(s));
    if (v & 2u) return fail(DGW_ETIMEOUT, "a work item waited too long for its instance's previous stage");
    if (v & 1u) return fail(DGW_ENONFINITE, "a stage produced a non-finite value");
    return DGW_OK;
}

extern "C" dgw_status dgw_batch_debug(dgw_batch* b, long long wait_limit, int unreachable)
{
    if (!b || wait_limit < 1) return fail(DGW_EINVAL, "bad arguments");
    b->wait_limit = wait_limit;
    b->unreachable = unreachable ? 1 : 0;
    return DGW_OK;
}

// ------------------------------------------------------------------------------------
// mass: sum_e |K_e| c_0^e by a fixed-order two-level tree
// ------------------------------------------------------------------------------------
template <typename Real>
__global__ void mass_partial_kernel(const Real* U0, int64_t E, double* partial)
{
    __shared__ double sh[kMassThreads];
    double s = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E;
         e += (int64_t)gridDim.x * blockDim.x)
        s += (double)U0[e];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

__global__ void mass_final_kernel(const double* partial, int n, double vol, double* out)
{
    __shared__ double sh[kMassThreads];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += partial[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0] * vol;
}

extern "C" dgw_status dgw_mass(dgw_ctx* c, const void* U, double* host_mass, void* stream)
{
    dgw_status st = check_ctx(c);
    if (st != DGW_OK) return st;
    if (!U || !host_mass) return fail(DGW_EINVAL, "NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    const double vol = c->mesh.dim == 1 ? c->h : c->h * c->h;
    if (c->params.prec == DGW_FP64)
        mass_partial_kernel<double><<<kMassBlocks, kMassThreads, 0, s>>>((const double*)U, c->E, c->partial);
    else
        mass_partial_kernel<float><<<kMassBlocks, kMassThreads, 0, s>>>((const float*)U, c->E, c->partial);
    DGW_CUDA(cudaGetLastError());
    mass_final_kernel<<<1, kMassThreads, 0, s>>>(c->partial, kMassBlocks, vol, c->mass_dev);
    DGW_CUDA(cudaGetLastError());
    DGW_CUDA(cudaMemcpyAsync(host_mass, c->mass_dev, sizeof(double), cudaMemcpyDeviceToHost, s));
    DGW_CUDA(cudaStreamSynchronize(s));
    return DGW_OK;
}

// ------------------------------------------------------------------------------------
// discrete adjoint
// ------------------------------------------------------------------------------------
static dgw_status adjoint_ready(dgw_ctx* c)
{
    for (int f = 0; f < 2 * c->mesh.dim; ++f)
        if (c->mesh.bc[f] != DGW_BC_PERIODIC)
            return fail(DGW_EUNSUPPORTED, "the adjoint is built for periodic meshes");
    if (c->flux.kind != DGW_FLUX_ADVECT && c->flux.kind != DGW_FLUX_BURGERS)
        return fail(DGW_EUNSUPPORTED, "the adjoint is built for the advection and Burgers fluxes");
    if (c->params.stab == DGW_STAB_ZHAO)
        return fail(DGW_EUNSUPPORTED, "the adjoint differentiates the DG, LO and WENO stabilizations");
    const size_t bytes = (size_t)c->K * c->E * c->eb;
    cudaError_t e = cudaSuccess;
    if (!c->adj_ws) e = cudaMalloc(&c->adj_ws, bytes);
    if (e == cudaSuccess && !c->adj_wn) e = cudaMalloc(&c->adj_wn, bytes * 2 * c->mesh.dim);
    if (e == cudaSuccess && !c->adj_b1) e = cudaMalloc(&c->adj_b1, bytes);
    if (e == cudaSuccess && !c->adj_b2) e = cudaMalloc(&c->adj_b2, bytes);
    if (e != cudaSuccess) return fail(DGW_ENOMEM, "adjoint buffers: %s", cudaGetErrorString(e));
    return DGW_OK;
}

// out = c0 x0 + c1 x1 + c2 x2 + cv J_L(U)^T lam
static cudaError_t vjp_combine(const dgw_ctx* c, const void* U, const void* lam, const void* x0, double c0,
                               const void* x1, double c1, const void* x2, double c2, double cv, void* out,
                               cudaStream_t s)
{
    StageArgs a = base_args(c);
    a.Uk = U;
    const bool f64 = c->params.prec == DGW_FP64;
    const int d = c->mesh.dim;
    cudaError_t e = f64 ? (d == 1 ? launch_vjp_f64_d1(a, c->p, c->flux.kind, lam, c->adj_ws, c->adj_wn, s)
                                  : launch_vjp_f64_d2(a, c->p, c->flux.kind, lam, c->adj_ws, c->adj_wn, s))
                        : (d == 1 ? launch_vjp_f32_d1(a, c->p, c->flux.kind, lam, c->adj_ws, c->adj_wn, s)
                                  : launch_vjp_f32_d2(a, c->p, c->flux.kind, lam, c->adj_ws, c->adj_wn, s));
    if (e != cudaSuccess) return e;
    GatherArgs g;
    std::memset(&g, 0, sizeof g);
    g.E = c->E; g.nx = c->mesh.nx; g.ny = d == 2 ? c->mesh.ny : 1;
    g.wself = c->adj_ws; g.wnb = c->adj_wn;
    g.x[0] = x0; g.x[1] = x1; g.x[2] = x2;
    g.coef[0] = c0; g.coef[1] = c1; g.coef[2] = c2;
    g.cvjp = cv;
    g.out = out;
    return f64 ? (d == 1 ? launch_gather_f64_d1(g, c->p, s) : launch_gather_f64_d2(g, c->p, s))
               : (d == 1 ? launch_gather_f32_d1(g, c->p, s) : launch_gather_f32_d2(g, c->p, s));
}

extern "C" dgw_status dgw_residual_vjp(dgw_ctx* c, const void* U, const void* lam, void* out, void* stream)
{
    dgw_status st = check_ctx(c);
    if (st != DGW_OK) return st;
    if (!U || !lam || !out) return fail(DGW_EINVAL, "NULL array");
    if (out == U || out == lam) return fail(DGW_EINVAL, "out must not overlap U or lam");
    st = adjoint_ready(c);
    if (st != DGW_OK) return st;
    DGW_CUDA(vjp_combine(c, U, lam, nullptr, 0.0, nullptr, 0.0, nullptr, 0.0, 1.0, out, (cudaStream_t)stream));
    return DGW_OK;
}

// Reverse of one SSP-RK3 step (Eq. ssp).  With a = lam^{n+1}:
//   lam_U2 = 2/3 a + 2/3 dt J_L(U2)^T a
//   lam_U1 = 1/4 lam_U2 + 1/4 dt J_L(U1)^T lam_U2
//   lam^n  = 1/3 a + 3/4 lam_U2 + lam_U1 + dt J_L(U^n)^T lam_U1
// where U1, U2 are recomputed from U^n.
extern "C" dgw_status dgw_adjoint_step(dgw_ctx* c, const void* U_n, const void* lam_np1, void* lam_n,
                                       double dt, void* stream)
{
    dgw_status st = check_ctx(c);
    if (st != DGW_OK) return st;
    if (!U_n || !lam_np1 || !lam_n) return fail(DGW_EINVAL, "NULL array");
    if (!std::isfinite(dt)) return fail(DGW_EINVAL, "dt must be finite");
    if (c->params.rk_order != 3)
        return fail(DGW_EUNSUPPORTED, "the adjoint step reverses the SSP-RK3 step (rk_order 3)");
    st = adjoint_ready(c);
    if (st != DGW_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    StageArgs a = base_args(c);
    a.Uk = U_n; a.Un = nullptr; a.Uout = c->S1;
    a.cn = 0.0; a.ck = 1.0; a.cl = dt;
    DGW_CUDA(launch(c, a, 0, s));
    a.Uk = c->S1; a.Un = U_n; a.Uout = c->S2;
    a.cn = 0.75; a.ck = 0.25; a.cl = 0.25 * dt;
    DGW_CUDA(launch(c, a, 0, s));
    DGW_CUDA(vjp_combine(c, c->S2, lam_np1, lam_np1, 2.0 / 3.0, nullptr, 0.0, nullptr, 0.0, 2.0 / 3.0 * dt,
                         c->adj_b1, s));
    DGW_CUDA(vjp_combine(c, c->S1, c->adj_b1, c->adj_b1, 0.25, nullptr, 0.0, nullptr, 0.0, 0.25 * dt,
                         c->adj_b2, s));
    DGW_CUDA(vjp_combine(c, U_n, c->adj_b2, lam_np1, 1.0 / 3.0, c->adj_b1, 0.75, c->adj_b2, 1.0, dt, lam_n, s));
    return DGW_OK;
}

extern "C" dgw_status dgw_rk_step_stages(dgw_ctx* c, const void* U, double dt, void* U1, void* U2, void* U_next,
                                         void* stream)
{
    dgw_status st = check_ctx(c);
    if (st != DGW_OK) return st;
    if (!U || !U1 || !U2) return fail(DGW_EINVAL, "NULL array");
    if (!aligned16(U) || !aligned16(U1) || !aligned16(U2) || (U_next && !aligned16(U_next)))
        return fail(DGW_EINVAL, "arrays must be 16-byte aligned");
    if (U1 == U || U2 == U || U1 == U2 || U_next == U1 || U_next == U2)
        return fail(DGW_EINVAL, "the stage states must not overlap U, U_next or each other");
    if (!std::isfinite(dt)) return fail(DGW_EINVAL, "dt must be finite");
    if (c->params.rk_order != 3) return fail(DGW_EUNSUPPORTED, "stage states of the SSP-RK3 step (rk_order 3)");
    if (c->state_sides) return fail(DGW_EUNSUPPORTED, "dgw_rk_step_stages keeps no time (prescribed-state sides)");
    cudaStream_t s = (cudaStream_t)stream;
    StageArgs a = base_args(c);
    a.Uk = U; a.Un = nullptr; a.Uout = U1;
    a.cn = 0.0; a.ck = 1.0; a.cl = dt;
    DGW_CUDA(launch(c, a, 0, s));
    a.Uk = U1; a.Un = U; a.Uout = U2;
    a.cn = 0.75; a.ck = 0.25; a.cl = 0.25 * dt;
    DGW_CUDA(launch(c, a, 0, s));
    if (U_next) {
        a.Uk = U2; a.Un = U; a.Uout = U_next;
        a.cn = 1.0 / 3.0; a.ck = 2.0 / 3.0; a.cl = 2.0 / 3.0 * dt;
        DGW_CUDA(launch(c, a, 0, s));
    }
    return DGW_OK;
}

extern "C" dgw_status dgw_adjoint_step_stages(dgw_ctx* c, const void* U_n, const void* U1, const void* U2,
                                              const void* lam_np1, void* lam_n, double dt, void* stream)
{
    dgw_status st = check_ctx(c);
    if (st != DGW_OK) return st;
    if (!U_n || !U1 || !U2 || !lam_np1 || !lam_n) return fail(DGW_EINVAL, "NULL array");
    if (!std::isfinite(dt)) return fail(DGW_EINVAL, "dt must be finite");
    if (c->params.rk_order != 3)
        return fail(DGW_EUNSUPPORTED, "the adjoint step reverses the SSP-RK3 step (rk_order 3)");
    st = adjoint_ready(c);
    if (st != DGW_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    DGW_CUDA(vjp_combine(c, U2, lam_np1, lam_np1, 2.0 / 3.0, nullptr, 0.0, nullptr, 0.0, 2.0 / 3.0 * dt,
                         c->adj_b1, s));
    DGW_CUDA(vjp_combine(c, U1, c->adj_b1, c->adj_b1, 0.25, nullptr, 0.0, nullptr, 0.0, 0.25 * dt,
                         c->adj_b2, s));
    DGW_CUDA(vjp_combine(c, U_n, c->adj_b2, lam_np1, 1.0 / 3.0, c->adj_b1, 0.75, c->adj_b2, 1.0, dt, lam_n, s));
    return DGW_OK;
}

template <typename Real>
__global__ void misfit_kernel(const Real* U, const Real* Ut, Real* grad, int64_t E, int K, int n1, int dim,
                              double h, double* partial)
{
    __shared__ double sh[kMassThreads];
    double s = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
        for (int k = 0; k < K; ++k) {
            const int i = k % n1, j = k / n1;
            double m = 0.5 * h * 2.0 / (2 * i + 1);            // mass of P_i on a cell of width h
            if (dim == 2) m *= 0.5 * h * 2.0 / (2 * j + 1);
            const double d = (double)U[k * E + e] - (double)Ut[k * E + e];
            s += 0.5 * m * d * d;
            if (grad) grad[k * E + e] = (Real)(m * d);
        }
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

extern "C" dgw_status dgw_misfit(dgw_ctx* c, const void* U, const void* U_target, double* host_J, void* grad,
                                 void* stream)
{
    dgw_status st = check_ctx(c);
    if (st != DGW_OK) return st;
    if (!U || !U_target || !host_J) return fail(DGW_EINVAL, "NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    if (c->params.prec == DGW_FP64)
        misfit_kernel<double><<<kMassBlocks, kMassThreads, 0, s>>>((const double*)U, (const double*)U_target,
                                                                   (double*)grad, c->E, c->K, c->p + 1, c->mesh.dim,
                                                                   c->h, c->partial);
    else
        misfit_kernel<float><<<kMassBlocks, kMassThreads, 0, s>>>((const float*)U, (const float*)U_target,
                                                                 (float*)grad, c->E, c->K, c->p + 1, c->mesh.dim,
                                                                 c->h, c->partial);
    DGW_CUDA(cudaGetLastError());
    mass_final_kernel<<<1, kMassThreads, 0, s>>>(c->partial, kMassBlocks, 1.0, c->mass_dev);
    DGW_CUDA(cudaGetLastError());
    DGW_CUDA(cudaMemcpyAsync(host_J, c->mass_dev, sizeof(double), cudaMemcpyDeviceToHost, s));
    DGW_CUDA(cudaStreamSynchronize(s));
    return DGW_OK;
}

extern "C" dgw_status dgw_sync_status(dgw_ctx* c, void* stream)
{
    dgw_status st = check_ctx(c);
    if (st != DGW_OK) return st;
    unsigned v = 0;
    cudaStream_t s = (cudaStream_t)stream;
    DGW_CUDA(cudaMemcpyAsync(&v, c->flag, sizeof v, cudaMemcpyDeviceToHost, s));
    DGW_CUDA(cudaMemsetAsync(c->flag, 0, sizeof(unsigned), s));
    DGW_CUDA(cudaStreamSynchronize(s));
    if (v & 2u) return fail(DGW_ETIMEOUT, "a stage kernel's bounded wait for its TMA copy gave up (its tile was skipped)");
    if (v & 1u) return fail(DGW_ENONFINITE, "a stage produced a non-finite value");
    return DGW_OK;
}

extern "C" dgw_status dgw_set_time(dgw_ctx* c, double t, void* stream)
{
    dgw_status st = check_ctx(c);
    if (st != DGW_OK) return st;
    if (!std::isfinite(t)) return fail(DGW_EINVAL, "t must be finite");
    cudaStream_t s = (cudaStream_t)stream;
    static thread_local double host_t;       // pageable source: the copy reads it before returning
    host_t = t;
    DGW_CUDA(cudaMemcpyAsync(c->t_dev, &host_t, sizeof(double), cudaMemcpyHostToDevice, s));
    DGW_CUDA(cudaStreamSynchronize(s));
    return DGW_OK;
}

extern "C" dgw_status dgw_get_time(dgw_ctx* c, double* t, void* stream)
{
    dgw_status st = check_ctx(c);
    if (st != DGW_OK) return st;
    if (!t) return fail(DGW_EINVAL, "NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    DGW_CUDA(cudaMemcpyAsync(t, c->t_dev, sizeof(double), cudaMemcpyDeviceToHost, s));
    DGW_CUDA(cudaStreamSynchronize(s));
    return DGW_OK;
}

extern "C" dgw_status dgw_debug(dgw_ctx* c, int wait_limit)
{
    dgw_status st = check_ctx(c);
    if (st != DGW_OK) return st;
    c->wait_limit = wait_limit;
    drop_graphs(c);          // the cached graphs hold the old launch parameters
    return DGW_OK;
}

extern "C" dgw_status dgw_set_stage_kernel(dgw_ctx* c, int choice)
{
    dgw_status st = check_ctx(c);
    if (st != DGW_OK) return st;
    if (choice < 0 || choice > 2) return fail(DGW_EINVAL, "stage kernel choice %d (0, 1 or 2)", choice);
    c->stage_kernel = choice;
    drop_graphs(c);          // the cached graphs hold the old kernels
    return DGW_OK;
}

// ------------------------------------------------------------------------------------
// self-test of the float sin/cos used by the KPP flux
// ------------------------------------------------------------------------------------
__global__ void sincos_selftest_kernel(const float* x, float* s, float* c, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dgw::fast_sincos(x[i], &s[i], &c[i]);
}

extern "C" dgw_status dgw_selftest_sincos(const float* x, float* s, float* c, int64_t n, void* stream)
{
    if (!x || !s || !c || n < 0) return fail(DGW_EINVAL, "bad arguments");
    if (n == 0) return DGW_OK;
    const int threads = 256;
    sincos_selftest_kernel<<<(unsigned)((n + threads - 1) / threads), threads, 0, (cudaStream_t)stream>>>(x, s, c, n);
    DGW_CUDA(cudaGetLastError());
    return DGW_OK;
}

extern "C" dgw_status dgw_selftest_tc_volume(const float* U, float* out, int64_t ntiles, int variant, float* ms,
                                             void* stream)
{
    if (!U || !out || ntiles < 0 || (variant != 0 && variant != 1)) return fail(DGW_EINVAL, "bad arguments");
    if (((uintptr_t)U & 15u) || ((uintptr_t)out & 15u)) return fail(DGW_EINVAL, "arrays must be 16-byte aligned");
    if (ntiles == 0) return DGW_OK;
    static std::mutex mu;
    static std::set<int> ready;                 // devices with the degree-3 float 2D tables
    int dev = -1;
    DGW_CUDA(cudaGetDevice(&dev));
    {
        std::lock_guard<std::mutex> lock(mu);
        if (!ready.count(dev)) {
            HostTables t;
            build_tables(3, &t);
            DGW_CUDA(upload_tables_f32_d2(t));
            ready.insert(dev);
        }
    }
    unsigned* flag = nullptr;
    DGW_CUDA(cudaMalloc(&flag, sizeof(unsigned)));
    cudaError_t e = cudaMemset(flag, 0, sizeof(unsigned));
    if (e == cudaSuccess) e = launch_tc_volume_f32_d2(U, out, ntiles, variant, flag, ms, (cudaStream_t)stream);
    unsigned v = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&v, flag, sizeof v, cudaMemcpyDeviceToHost);
    cudaFree(flag);
    if (e != cudaSuccess) return fail(DGW_ECUDA, "tensor-core volume probe: %s", cudaGetErrorString(e));
    if (v & 2u) return fail(DGW_ETIMEOUT, "tensor-core volume probe: a bounded wait for the MMAs gave up");
    return DGW_OK;
}

// ------------------------------------------------------------------------------------
// SSP-RK3 steps without any device allocation
// ------------------------------------------------------------------------------------
// Some callers cannot call cudaMalloc: applications whose device memory is all owned by
// another allocator, and real-time code that allows no allocation after start-up (an
// allocation can block or fail at an arbitrary point).  dgw_rk_step_noalloc serves them:
// instead of a context's
// stage buffers it keeps the two SSP-RK3 stage states in this fixed array, which every
// GPU that loads the library holds until the process exits.  Layout: stage 1, stage 2
// (kNoAllocStageBytes each), then the kernels' error flag.  Nothing in it has to start
// at zero: each stage buffer is written in full before it is read, and the flag is
// only ever set.
static const size_t kNoAllocStageBytes = (size_t)8 << 20;   // 8 MiB per stage state
static __device__ __align__(256) unsigned char g_noalloc_scratch[2 * kNoAllocStageBytes + 256];

static std::mutex g_noalloc_mu;
static std::map<int, unsigned char*> g_noalloc_addr;        // device -> array address
static std::set<std::tuple<int, int, int, int>> g_noalloc_tables;   // device, prec, dim, p

extern "C" dgw_status dgw_rk_step_noalloc(const dgw_mesh* mesh, int p, const dgw_flux* flux,
                                          const dgw_params* params, void* U, double dt,
                                          int nsteps, void* stream)
{
    if (!mesh || !flux || !params || !U) return fail(DGW_EINVAL, "NULL argument to dgw_rk_step_noalloc");
    const dgw_mesh& m = *mesh;
    if (m.dim != 1 && m.dim != 2) return fail(DGW_EINVAL, "dim must be 1 or 2");
    if (m.nx < 1 || (m.dim == 2 && m.ny < 1)) return fail(DGW_EINVAL, "nx, ny must be >= 1");
    if (!(m.x1 > m.x0) || (m.dim == 2 && !(m.y1 > m.y0))) return fail(DGW_EINVAL, "empty box");
    for (int f = 0; f < 2 * m.dim; ++f)
        if (m.bc[f] < DGW_BC_PERIODIC || m.bc[f] > DGW_BC_OUTFLOW) return fail(DGW_EINVAL, "bad bc[%d]", f);
    for (int a = 0; a < m.dim; ++a)
        if ((m.bc[2 * a] == DGW_BC_PERIODIC) != (m.bc[2 * a + 1] == DGW_BC_PERIODIC))
            return fail(DGW_EINVAL, "periodic sides must come in pairs");
    const double hx = (m.x1 - m.x0) / m.nx;
    if (m.dim == 2 && std::fabs(hx - (m.y1 - m.y0) / m.ny) > 1e-12 * hx)
        return fail(DGW_EUNSUPPORTED, "2D cells must be square");
    if (p < 1 || p > kMaxP) return fail(DGW_EUNSUPPORTED, "degree p=%d not built (1..3)", p);
    if (flux->kind == DGW_FLUX_EULER) return fail(DGW_EUNSUPPORTED, "dgw_rk_step_noalloc is built for the scalar laws");
    if (flux->kind < DGW_FLUX_ADVECT || flux->kind > DGW_FLUX_KPP) return fail(DGW_EINVAL, "bad flux kind");
    if (!(flux->lambda_nu >= 0.0)) return fail(DGW_EINVAL, "lambda_nu must be >= 0");
    dgw_status st = check_params(params, m.dim);
    if (st != DGW_OK) return st;
    if (!aligned16(U)) return fail(DGW_EINVAL, "U must be 16-byte aligned");
    if (nsteps < 0) return fail(DGW_EINVAL, "nsteps < 0");
    if (!std::isfinite(dt)) return fail(DGW_EINVAL, "dt must be finite");
    const int64_t E = m.dim == 1 ? (int64_t)m.nx : (int64_t)m.nx * m.ny;
    const int K = m.dim == 1 ? p + 1 : (p + 1) * (p + 1);
    const int eb = params->prec == DGW_FP64 ? 8 : 4;
    const double bytes = (double)K * (double)E * eb;
    if (bytes > (double)kNoAllocStageBytes)
        return fail(DGW_EINVAL,
                    "dgw_rk_step_noalloc: a state of %.0f bytes exceeds the fixed stage capacity of %zu "
                    "bytes (K*E*elem_bytes); use dgw_create/dgw_rk_step for larger meshes",
                    bytes, kNoAllocStageBytes);
    if (nsteps == 0) return DGW_OK;

    int dev = -1;
    DGW_CUDA(cudaGetDevice(&dev));
    unsigned char* base = nullptr;
    {
        // once per device (with that device current): the array's device address, and
        // the operator tables of this precision, dimension and degree
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        auto it = g_noalloc_addr.find(dev);
        if (it == g_noalloc_addr.end()) {
            void* ptr = nullptr;
            DGW_CUDA(cudaGetSymbolAddress(&ptr, g_noalloc_scratch));
            it = g_noalloc_addr.emplace(dev, static_cast<unsigned char*>(ptr)).first;
        }
        base = it->second;
        const auto key = std::make_tuple(dev, params->prec, m.dim, p);
        if (!g_noalloc_tables.count(key)) {
            HostTables t;
            build_tables(p, &t);
            cudaError_t ce;
            if (params->prec == DGW_FP64) ce = m.dim == 1 ? upload_tables_f64_d1(t) : upload_tables_f64_d2(t);
            else ce = m.dim == 1 ? upload_tables_f32_d1(t) : upload_tables_f32_d2(t);
            if (ce != cudaSuccess) return fail(DGW_ECUDA, "table upload: %s", cudaGetErrorString(ce));
            g_noalloc_tables.insert(key);
        }
    }

    // A context that lives on the host stack and points into the fixed array.
    dgw_ctx c;
    c.device = dev;
    c.mesh = m;
    if (m.dim == 1) c.mesh.ny = 1;
    c.p = p;
    c.flux = *flux;
    c.params = *params;
    c.K = K;
    c.E = E;
    c.eb = eb;
    c.h = hx;
    c.S1 = base;
    c.S2 = base + kNoAllocStageBytes;
    c.flag = reinterpret_cast<unsigned*>(base + 2 * kNoAllocStageBytes);
    DGW_CUDA(enqueue_steps(&c, U, dt, nsteps, (cudaStream_t)stream));
    return DGW_OK;
}

extern "C" const char* dgw_last_error(void) { return g_err.c_str(); }

extern "C" const char* dgw_version(void) { return "dgw 0.1 (sm_103a)"; }
