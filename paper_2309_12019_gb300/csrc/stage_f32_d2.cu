// Stage kernels, float precision, 2D.
#define DGW_REAL float
#define DGW_DIM 2
#define DGW_NS f32_d2
#define DGW_TC_VOLUME 1
#include "dgw_stage_impl.cuh"

namespace dgw {
cudaError_t launch_stage_f32_d2(const StageArgs& a, int p, int flux, int mode, cudaStream_t s)
{
    return f32_d2::launch(a, p, flux, mode, s);
}
cudaError_t launch_batch_f32_d2(const BatchArgs& a, int p, int rows, int grid, cudaStream_t s)
{
    return f32_d2::launch_batch(a, p, rows, grid, s);
}
int batch_blocks_per_sm_f32_d2(int p, int rows) { return f32_d2::batch_blocks_per_sm(p, rows); }
bool batch_rows_built_f32_d2(int rows) { return f32_d2::batch_rows_built(rows); }
cudaError_t launch_vjp_f32_d2(const StageArgs& a, int p, int flux, const void* lam, void* ws, void* wn, cudaStream_t s)
{
    return f32_d2::launch_vjp(a, p, flux, lam, ws, wn, s);
}
cudaError_t launch_gather_f32_d2(const GatherArgs& g, int p, cudaStream_t s) { return f32_d2::launch_gather(g, p, s); }
cudaError_t upload_tables_f32_d2(const HostTables& t) { return f32_d2::upload_tables(t); }
cudaError_t launch_tc_volume_f32_d2(const float* U, float* out, int64_t ntiles, int variant, unsigned* flag,
                                    float* ms, cudaStream_t s)
{
    return f32_d2::launch_tc_volume(U, out, ntiles, variant, flag, ms, s);
}
}  // namespace dgw
