// Stage kernels, double precision, 1D.
#define DGW_REAL double
#define DGW_DIM 1
#define DGW_NS f64_d1
#include "dgw_stage_impl.cuh"

namespace dgw {
cudaError_t launch_stage_f64_d1(const StageArgs& a, int p, int flux, int mode, cudaStream_t s)
{
    return f64_d1::launch(a, p, flux, mode, s);
}
cudaError_t launch_batch_f64_d1(const BatchArgs& a, int p, int rows, int grid, cudaStream_t s)
{
    return f64_d1::launch_batch(a, p, rows, grid, s);
}
int batch_blocks_per_sm_f64_d1(int p, int rows) { return f64_d1::batch_blocks_per_sm(p, rows); }
bool batch_rows_built_f64_d1(int rows) { return f64_d1::batch_rows_built(rows); }
cudaError_t launch_vjp_f64_d1(const StageArgs& a, int p, int flux, const void* lam, void* ws, void* wn, cudaStream_t s)
{
    return f64_d1::launch_vjp(a, p, flux, lam, ws, wn, s);
}
cudaError_t launch_gather_f64_d1(const GatherArgs& g, int p, cudaStream_t s) { return f64_d1::launch_gather(g, p, s); }
cudaError_t upload_tables_f64_d1(const HostTables& t) { return f64_d1::upload_tables(t); }
}  // namespace dgw
