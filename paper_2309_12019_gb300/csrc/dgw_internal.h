// Internal declarations shared by the translation units of libdgw (not part of the ABI).
#pragma once

#include <cstdint>

#include <cuda.h>
#include <cuda_runtime.h>

namespace dgw {

constexpr int kMaxP = 3;
constexpr int kMaxN1 = kMaxP + 1;          // modes per direction
constexpr int kMaxNQ = kMaxP + 2;          // Gauss points per direction (p + 2)
constexpr int kMaxK = kMaxN1 * kMaxN1;     // modes per element (2D)

// 2D tiles are kTileX2 threads wide.  The batch kernel runs 2, 4 or 8 (float; double:
// kTileY2) thread rows of one cell each, the height picked per degree by its autotuner.
// The stage kernel runs stage_thread_rows() rows, and in float a thread
// advances two cells stacked in y (their arithmetic paired on the packed FP32 pipe), so a
// stage tile spans kTileX2 x stage_rows() cells.  Its TMA box spans kTileX2 + 8 columns
// (the halo column on each side, widened so the box starts on a 16-byte boundary) and
// stage_rows() + 2 rows, for all K modes.
constexpr int kTileX2 = 32;
constexpr int kTileY2 = 4;
constexpr int kBoxX2 = kTileX2 + 8;
constexpr int stage_lanes(bool f64) { return f64 ? 1 : 2; }
constexpr int stage_thread_rows(bool f64) { return f64 ? kTileY2 : 2 * kTileY2; }
constexpr int stage_rows(bool f64) { return stage_thread_rows(f64) * stage_lanes(f64); }
// The persistent float stage kernel (whole-mesh launches): one CTA of 512 threads per SM
// walks tiles of kTileX2 x kPRows cells; its boxes are kBoxX2 x (kPRows + 2) x K (Uk) and
// kTileX2 x kPRows x K (Un).
constexpr int kPRows = 32;

enum : int { BC_PERIODIC = 0, BC_INFLOW_ZERO = 1, BC_OUTFLOW = 2, BC_REFLECT = 3, BC_STATE = 4 };
enum : int { FLUX_ADVECT = 0, FLUX_ROTATION = 1, FLUX_BURGERS = 2, FLUX_KPP = 3, FLUX_EULER = 4 };
enum : int { STAB_DG = 0, STAB_LO = 1, STAB_WENO = 2, STAB_ZHAO = 3 };

// Operator tables of degree p, built once in double on the host (dgw_tables.cu) and
// rounded to the kernel precision when uploaded.  Reference element [-1, 1]^d.
struct HostTables {
    int p;
    double g[kMaxNQ];               // Gauss-Legendre nodes, p + 2 points
    double w[kMaxNQ];               // and weights
    double B[kMaxNQ][kMaxN1];       // P_i(g_q)
    double D[kMaxNQ][kMaxN1];       // P_i'(g_q)
    double T[2][kMaxN1][kMaxN1];    // T[s][i][m]: coefficient of P_i in P_m(xi + 2) (s = 0:
                                    // neighbour on the minus side) or P_m(xi - 2) (s = 1)
    double G1[kMaxN1][kMaxN1];      // seminorm Gram matrix, 1D
    double G2[kMaxK][kMaxK];        // seminorm Gram matrix, 2D (mode k = i + (p+1) j)
    double A1[kMaxN1][kMaxN1];      // int P_i' P_m'
    double A0[kMaxN1];              // int P_i^2 = 2 / (2i + 1)
    double minv[kMaxN1];            // (2i + 1) / 2
};

void build_tables(int p, HostTables* t);
void gauss_rule_public(int n, double* x, double* w);

// Arguments of one stage launch: Uout = cn*Un + ck*Uk + cl*L(Uk), where L is the
// stabilized DG right-hand side of Uk.  Pointers are of the kernel precision.
struct StageArgs {
    const void* Uk;
    const void* Un;        // may be null when cn == 0
    void* Uout;            // may be null in sensor-only launches
    double cn, ck, cl;
    int64_t E;
    int nx, ny;
    double x0, y0, h;
    int bc[4];
    double a0, a1, cx, cy, omega, lambda_nu;
    int stab;
    double q, b, w_nbr, eps_w, eps_s, theta;
    double gas_gamma;      // Euler system: ratio of heat capacities
    double* gamma_out;     // optional per-element gamma (double)
    unsigned* flag;        // bit 0: non-finite output; bit 1 (value 2): a bounded wait gave up
    const CUtensorMap* tmap;   // 2D: TMA descriptor of Uk (box kBoxX2 x (stage_rows + 2) x K), or null
    const CUtensorMap* tmap_un;  // 2D: TMA descriptor of Un (box kTileX2 x stage_rows x K), or null
    const CUtensorMap* tmap_p;   // 2D float: descriptor of Uk for the persistent kernel (box kBoxX2 x
                                 // (kPRows + 2) x K), or null: that kernel runs only when given
    const CUtensorMap* tmap_un_p;  // and of Un (box kTileX2 x kPRows x K), or null
    int kernel_choice;     // whole-mesh float 2D stages: 0 automatic, 1 tile kernel, 2 persistent kernel
    int tile_row0;         // 2D: first tile row of the launch
    int tile_rows;         // 2D: tile rows of the launch (0: through the last row of the mesh)
    int wait_limit;        // polls of a bounded TMA wait: 0 the default limit, < 0 none (the
                           // wait gives up at once; diagnostic)
    // prescribed-state sides (2D Euler, DGW_BC_STATE): the stage's time is *t_dev + t_off
    const double* t_dev;
    double t_off;
    double bstate[2][4];
    double bsplit[4], bspeed[4];
    int bbelow[4], babove[4];
};

// ------------------------------------------------------------------------------------
// Batched ensemble: many independent meshes advanced by one persistent kernel per
// dimension and degree.  Work item = (stage, instance, chunk of tiles); an item waits
// only for its own instance's previous stage (per-instance counters, bounded spin).
// ------------------------------------------------------------------------------------
struct BatchInst {
    int64_t off;           // first coefficient of the instance in the packed state
    int64_t E;
    int nx, ny, p, flux;
    int ntx, ntiles;       // tiles per row, tiles per stage
    int bc[4];
    double x0, y0, h, a0, a1, cx, cy, omega, lambda_nu, dt;
};

struct BatchItem {
    int inst, tile0, ntile, pad;
};

struct BatchArgs {
    const BatchInst* inst;
    const BatchItem* items;
    int nitems;
    int nstages;                   // 3 * steps
    void* U;
    void* S1;
    void* S2;
    unsigned long long* queue;     // dequeue counter, zero at launch
    unsigned long long* done;      // per instance: tiles finished, zero at launch
    unsigned* flag;                // bit 0: non-finite; bit 1: a bounded wait gave up
    int* abort;                    // set when a wait gave up: every CTA stops
    int stab;
    double q, b, w_nbr, eps_w, eps_s, theta;
    long long wait_limit;          // spin iterations before a wait gives up
    int unreachable;               // diagnostic: ask one tile more than exists (wait must give up)
};

// Discrete adjoint: out = sum_i coef[i] x[i] + cvjp * J_L(U)^T lam, the transpose-Jacobian
// product assembled from per-cell partials (wself: own, wnb: one block per face).
struct GatherArgs {
    int64_t E;
    int nx, ny;
    const void* wself;
    const void* wnb;
    const void* x[3];      // may be null
    double coef[3];
    double cvjp;
    void* out;
};

// Launchers, one per (precision, dimension) translation unit.  mode 0: stage or
// residual; mode 1: sensor only (writes gamma_out).
cudaError_t launch_stage_f32_d1(const StageArgs& a, int p, int flux, int mode, cudaStream_t s);
cudaError_t launch_stage_f32_d2(const StageArgs& a, int p, int flux, int mode, cudaStream_t s);
cudaError_t launch_stage_f64_d1(const StageArgs& a, int p, int flux, int mode, cudaStream_t s);
cudaError_t launch_stage_f64_d2(const StageArgs& a, int p, int flux, int mode, cudaStream_t s);

// Batch kernels per (degree p, tile height `rows`): 2D float tiles of 2, 4 or 8 cell rows,
// 2D double tiles of kTileY2, 1D tiles of one row (batch_rows_built_*).
cudaError_t launch_batch_f32_d1(const BatchArgs& a, int p, int rows, int grid, cudaStream_t s);
cudaError_t launch_batch_f32_d2(const BatchArgs& a, int p, int rows, int grid, cudaStream_t s);
cudaError_t launch_batch_f64_d1(const BatchArgs& a, int p, int rows, int grid, cudaStream_t s);
cudaError_t launch_batch_f64_d2(const BatchArgs& a, int p, int rows, int grid, cudaStream_t s);
int batch_blocks_per_sm_f32_d1(int p, int rows);
int batch_blocks_per_sm_f32_d2(int p, int rows);
int batch_blocks_per_sm_f64_d1(int p, int rows);
int batch_blocks_per_sm_f64_d2(int p, int rows);
bool batch_rows_built_f32_d1(int rows);
bool batch_rows_built_f32_d2(int rows);
bool batch_rows_built_f64_d1(int rows);
bool batch_rows_built_f64_d2(int rows);

cudaError_t launch_vjp_f32_d1(const StageArgs& a, int p, int flux, const void* lam, void* ws, void* wn, cudaStream_t s);
cudaError_t launch_vjp_f32_d2(const StageArgs& a, int p, int flux, const void* lam, void* ws, void* wn, cudaStream_t s);
cudaError_t launch_vjp_f64_d1(const StageArgs& a, int p, int flux, const void* lam, void* ws, void* wn, cudaStream_t s);
cudaError_t launch_vjp_f64_d2(const StageArgs& a, int p, int flux, const void* lam, void* ws, void* wn, cudaStream_t s);
cudaError_t launch_gather_f32_d1(const GatherArgs& g, int p, cudaStream_t s);
cudaError_t launch_gather_f32_d2(const GatherArgs& g, int p, cudaStream_t s);
cudaError_t launch_gather_f64_d1(const GatherArgs& g, int p, cudaStream_t s);
cudaError_t launch_gather_f64_d2(const GatherArgs& g, int p, cudaStream_t s);

// The Q3 KPP volume term on 128-cell tiles: variant 0 on the CUDA cores (packed FP32),
// 1 on the tensor cores (tcgen05, three TF32 passes).  Synchronous; *ms (may be NULL)
// receives the kernel's duration from CUDA events on the stream.  Diagnostic.
cudaError_t launch_tc_volume_f32_d2(const float* U, float* out, int64_t ntiles, int variant, unsigned* flag,
                                    float* ms, cudaStream_t s);

cudaError_t upload_tables_f32_d1(const HostTables& t);
cudaError_t upload_tables_f32_d2(const HostTables& t);
cudaError_t upload_tables_f64_d1(const HostTables& t);
cudaError_t upload_tables_f64_d2(const HostTables& t);

}  // namespace dgw
