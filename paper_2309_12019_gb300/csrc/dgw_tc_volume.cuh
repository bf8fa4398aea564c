// Volume term of the KPP problem at Q3 on tensor cores: a measurement of the alternative
// to the stage kernel's packed-FP32 contractions (included by the float 2D stage unit).
//
// The volume term of a cell (Eq. weak2) is two contractions around the flux:
//   u_n   = sum_k B1[n][k] c_k        (k = i + 4 j modes, n = qx + 5 qy Gauss points)
//   acc_k = sum_n B2[k][n] F_n        (F = (sin u, cos u) at the 25 points: 50 values)
// with B1[n][k] = P_i(g_qx) P_j(g_qy), B2[k][n] = W_qx W_qy P_i'(g_qx) P_j(g_qy) for the
// x-flux and W_qx W_qy P_i(g_qx) P_j'(g_qy) for the y-flux.  Over a tile of 128 cells
// these are the GEMMs [128 x 16] x [16 x 25] and [128 x 50] x [50 x 16].
//
// tc_volume_kernel: one CTA per tile at a time (persistent), 128 threads, thread = cell =
// TMEM lane.  Each operand is split into TF32 parts, x = hi + lo with hi = x with its low
// 13 mantissa bits cleared, and each product taken as hi.hi + hi.lo + lo.hi (three
// tcgen05.mma kind::tf32 passes, FP32 accumulation in TMEM), which keeps about 2^-21 of
// relative accuracy (one pass keeps 2^-11).  Operands sit in shared memory in the
// no-swizzle K-major layout: core matrices of 8 rows x 16 bytes, 128 bytes between the two
// core matrices of one 8-element K slice, 256 bytes between groups of 8 rows.
// cc_volume_kernel: the same function on the CUDA cores, as the stage kernel computes it
// (two cells per thread on packed FP32, symmetric-node contractions, one row at a time).

namespace tcv {
constexpr int M = 128;              // cells per tile
constexpr int K1 = 16, N1P = 32;    // modes; Gauss points 25, padded to an MMA width
constexpr int K2 = 56, N2 = 16;     // 50 flux values padded to 7 slices of 8; modes
constexpr int A1_BYTES = M * K1 * 4, A2_BYTES = M * K2 * 4;
constexpr int B1_BYTES = N1P * K1 * 4, B2_BYTES = N2 * K2 * 4;
constexpr int B_BYTES = 2 * (B1_BYTES + B2_BYTES);      // hi and lo parts of both tables
// shared memory: A1 hi/lo, A2 hi/lo, B (copied in once), the mbarrier and the TMEM address
constexpr int OFF_A1H = 0, OFF_A1L = OFF_A1H + A1_BYTES, OFF_A2H = OFF_A1L + A1_BYTES,
              OFF_A2L = OFF_A2H + A2_BYTES, OFF_B = OFF_A2L + A2_BYTES, OFF_BAR = OFF_B + B_BYTES,
              SMEM_BYTES = OFF_BAR + 16;
constexpr int TMEM_COLS = 64;       // D1 in columns 0..31, D2 in 32..47

// byte offset of element (row r, column k) of a K-major operand of `rows` rows
__host__ __device__ constexpr int koff(int r, int k, int rows)
{
    return (k / 8) * rows * 32 + (r / 8) * 256 + ((k % 8) / 4) * 128 + (r % 8) * 16 + (k % 4) * 4;
}
}  // namespace tcv

__device__ __forceinline__ float tf32_hi(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

// descriptor of a K-major, no-swizzle operand slice at shared address addr
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr)
{
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(256 >> 4) << 32) |
           (1ull << 46);
}

// instruction descriptor: D in FP32, A and B TF32, both K-major, M = 128
__host__ __device__ constexpr uint32_t umma_idesc_tf32(int n)
{
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(tcv::M >> 4) << 24);
}

__device__ __forceinline__ void umma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, int accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
        :: "r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(accumulate) : "memory");
}

__global__ void __launch_bounds__(128, 1) tc_volume_kernel(const float* __restrict__ U, float* __restrict__ out,
                                                            const unsigned char* __restrict__ Btab, int64_t ntiles,
                                                            unsigned* flag)
{
    using namespace tcv;
    extern __shared__ __align__(1024) unsigned char sm[];
    const int tid = threadIdx.x, warp = tid >> 5;
    const uint32_t base = (uint32_t)__cvta_generic_to_shared(sm);
    const uint32_t bar = base + OFF_BAR;
    uint32_t* taddr_s = reinterpret_cast<uint32_t*>(sm + OFF_BAR + 8);
    // the tables (hi and lo of B1 and B2, already in the operand layout) into shared memory
    for (int i = tid; i < B_BYTES / 16; i += blockDim.x)
        reinterpret_cast<uint4*>(sm + OFF_B)[i] = reinterpret_cast<const uint4*>(Btab)[i];
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(bar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"((uint32_t)__cvta_generic_to_shared(taddr_s)), "n"(TMEM_COLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *taddr_s;
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
    uint32_t phase = 0;
    bool failed = false;

    // bounded wait for the commit of the given parity; the CTA agrees on the outcome
    // (__syncthreads_or), so that no thread leaves the tile loop alone
    auto wait_mma = [&](uint32_t par) -> bool {
        bool ok = false;
        for (int it = 0; it < (1 << 22) && !ok; ++it) {
            uint32_t done;
            asm volatile("{\n\t.reg .pred p;\n\t"
                         "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                         "selp.u32 %0, 1, 0, p;\n\t}"
                         : "=r"(done) : "r"(bar), "r"(par) : "memory");
            ok = done != 0;
        }
        return __syncthreads_or(!ok) == 0;
    };
    auto commit = [&]() {
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                     :: "r"(bar) : "memory");
    };

    for (int64_t t = blockIdx.x; t < ntiles && !failed; t += gridDim.x) {
        const int64_t cell = t * M + tid;
        const int64_t ncell = ntiles * M;
        // 1. the cell's 16 coefficients, split, into row tid of A1
#pragma unroll
        for (int k = 0; k < K1; ++k) {
            const float x = U[(int64_t)k * ncell + cell];
            const float hi = tf32_hi(x);
            *reinterpret_cast<float*>(sm + OFF_A1H + koff(tid, k, M)) = hi;
            *reinterpret_cast<float*>(sm + OFF_A1L + koff(tid, k, M)) = tf32_hi(x - hi);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // 2. u = A1 B1^T: hi.hi + hi.lo + lo.hi over the two K slices
        if (tid == 0) {
            const uint32_t id = umma_idesc_tf32(N1P);
            const uint32_t a[2] = {base + OFF_A1H, base + OFF_A1L};
            const uint32_t b[2] = {base + OFF_B, base + OFF_B + B1_BYTES};
            const int pa[3] = {0, 0, 1}, pb[3] = {0, 1, 0};
            int n = 0;
#pragma unroll
            for (int pass = 0; pass < 3; ++pass)
#pragma unroll
                for (int s = 0; s < K1 / 8; ++s, ++n)
                    umma_tf32(tmem, umma_desc(a[pa[pass]] + s * M * 32), umma_desc(b[pb[pass]] + s * N1P * 32), id, n > 0);
            commit();
        }
        if (!wait_mma(phase)) { failed = true; break; }
        phase ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        uint32_t r[32];
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                     "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                     : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                       "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                       "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                       "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                       "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                     : "r"(lane_base) : "memory");
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        // 3. the flux at the 25 points, split, into row tid of A2 (x-flux, y-flux, zeros)
#pragma unroll
        for (int n = 0; n < 25; ++n) {
            float s, c;
            fast_sincos(__uint_as_float(r[n]), &s, &c);
            const float sh = tf32_hi(s), ch = tf32_hi(c);
            *reinterpret_cast<float*>(sm + OFF_A2H + koff(tid, n, M)) = sh;
            *reinterpret_cast<float*>(sm + OFF_A2L + koff(tid, n, M)) = tf32_hi(s - sh);
            *reinterpret_cast<float*>(sm + OFF_A2H + koff(tid, 25 + n, M)) = ch;
            *reinterpret_cast<float*>(sm + OFF_A2L + koff(tid, 25 + n, M)) = tf32_hi(c - ch);
        }
#pragma unroll
        for (int n = 50; n < K2; ++n) {
            *reinterpret_cast<float*>(sm + OFF_A2H + koff(tid, n, M)) = 0.f;
            *reinterpret_cast<float*>(sm + OFF_A2L + koff(tid, n, M)) = 0.f;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // 4. acc = A2 B2^T over seven K slices, three passes, into columns 32..47
        if (tid == 0) {
            const uint32_t id = umma_idesc_tf32(N2);
            const uint32_t a[2] = {base + OFF_A2H, base + OFF_A2L};
            const uint32_t b[2] = {base + OFF_B + 2 * B1_BYTES, base + OFF_B + 2 * B1_BYTES + B2_BYTES};
            const int pa[3] = {0, 0, 1}, pb[3] = {0, 1, 0};
            int n = 0;
#pragma unroll
            for (int pass = 0; pass < 3; ++pass)
#pragma unroll
                for (int s = 0; s < K2 / 8; ++s, ++n)
                    umma_tf32(tmem + 32, umma_desc(a[pa[pass]] + s * M * 32), umma_desc(b[pb[pass]] + s * N2 * 32), id, n > 0);
            commit();
        }
        if (!wait_mma(phase)) { failed = true; break; }
        phase ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        uint32_t q[16];
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                     : "=r"(q[0]), "=r"(q[1]), "=r"(q[2]), "=r"(q[3]), "=r"(q[4]), "=r"(q[5]), "=r"(q[6]), "=r"(q[7]),
                       "=r"(q[8]), "=r"(q[9]), "=r"(q[10]), "=r"(q[11]), "=r"(q[12]), "=r"(q[13]), "=r"(q[14]),
                       "=r"(q[15])
                     : "r"(lane_base + 32) : "memory");
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int k = 0; k < N2; ++k) out[(int64_t)k * ncell + cell] = __uint_as_float(q[k]);
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    if (failed) {
        // a wait gave up: report it, let the MMAs in flight finish (bounded), free TMEM
        if (tid == 0) atomicOr(flag, 2u);
        wait_mma(phase);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "n"(TMEM_COLS) : "memory");
}

// The same volume term on the CUDA cores: two cells per thread (cells c and c + 128 of a
// 256-cell block), the stage kernel's row loop (symmetric nodes, packed FP32).
__global__ void __launch_bounds__(128) cc_volume_kernel(const float* __restrict__ U, float* __restrict__ out,
                                                         int64_t ncell)
{
    constexpr int P = 3, N1 = 4, NQ = 5, K = 16;
    const Tab<P>& T = tab<P>();
    const int64_t c0 = (int64_t)blockIdx.x * 256 + threadIdx.x, c1 = c0 + 128;
    if (c0 >= ncell) return;
    const bool has1 = c1 < ncell;
    float2 c[K], acc[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        c[k] = make_float2(U[(int64_t)k * ncell + c0], has1 ? U[(int64_t)k * ncell + c1] : 0.f);
        acc[k] = make_float2(0.f, 0.f);
    }
#pragma unroll 1
    for (int qy = 0; qy < NQ; ++qy) {
        float2 rr[N1];
#pragma unroll
        for (int i = 0; i < N1; ++i) {
            float2 e = c[i];
#pragma unroll
            for (int j = 1; j < N1; ++j) e = vfma(T.B[qy][j], c[i + N1 * j], e);
            rr[i] = e;
        }
        float2 u[NQ], fx[NQ], fy[NQ];
        interp_sym<N1, NQ>(T.B, rr, u);
#pragma unroll
        for (int qx = 0; qx < NQ; ++qx) fast_sincos2(u[qx], &fx[qx], &fy[qx]);
        float2 px[N1], py[N1];
        project_sym<true, N1, NQ>(T.WD, fx, px);
        project_sym<false, N1, NQ>(T.WB, fy, py);
#pragma unroll
        for (int j = 0; j < N1; ++j)
#pragma unroll
            for (int i = 0; i < N1; ++i) {
                float2 t = acc[i + N1 * j];
                if (i > 0) t = vfma(T.WB[qy][j], px[i], t);
                if (j > 0) t = vfma(T.WD[qy][j], py[i], t);
                acc[i + N1 * j] = t;
            }
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
        out[(int64_t)k * ncell + c0] = acc[k].x;
        if (has1) out[(int64_t)k * ncell + c1] = acc[k].y;
    }
}

// Host: the tables B1 (25 x 16) and B2 (16 x 50) from the degree-3 tables, split into TF32
// hi and lo parts, in the operand layout (hi B1, lo B1, hi B2, lo B2).
static void tc_volume_tables(const HostTables& h, std::vector<unsigned char>& buf)
{
    using namespace tcv;
    buf.assign(B_BYTES, 0);
    auto put = [&](int off, int rows, int r, int k, double v) {
        const float x = (float)v;
        uint32_t ux;
        std::memcpy(&ux, &x, 4);
        ux &= 0xFFFFE000u;
        float hi;
        std::memcpy(&hi, &ux, 4);
        float lo = x - hi;
        uint32_t ul;
        std::memcpy(&ul, &lo, 4);
        ul &= 0xFFFFE000u;
        std::memcpy(&lo, &ul, 4);
        std::memcpy(&buf[off + koff(r, k, rows)], &hi, 4);
        std::memcpy(&buf[off + (rows == N1P ? B1_BYTES : B2_BYTES) + koff(r, k, rows)], &lo, 4);
    };
    for (int qy = 0; qy < 5; ++qy)
        for (int qx = 0; qx < 5; ++qx)
            for (int j = 0; j < 4; ++j)
                for (int i = 0; i < 4; ++i) {
                    const int n = qx + 5 * qy, k = i + 4 * j;
                    put(0, N1P, n, k, h.B[qx][i] * h.B[qy][j]);
                    const double w = h.w[qx] * h.w[qy];
                    put(2 * B1_BYTES, N2, k, n, w * h.D[qx][i] * h.B[qy][j]);
                    put(2 * B1_BYTES, N2, k, 25 + n, w * h.B[qx][i] * h.D[qy][j]);
                }
}

// The variant's kernel on stream st, bracketed by two events whose elapsed time goes to
// *ms.  The tensor-core tables are built once per device.  Synchronous.
static cudaError_t launch_tc_volume(const float* U, float* out, int64_t ntiles, int variant, unsigned* flag,
                                    float* ms, cudaStream_t st)
{
    static std::mutex mu;
    static std::map<int, unsigned char*> tables;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    unsigned char* dtab = nullptr;
    if (e == cudaSuccess && variant == 1) {
        std::lock_guard<std::mutex> lock(mu);
        auto it = tables.find(dev);
        if (it == tables.end()) {
            HostTables h;
            build_tables(3, &h);
            std::vector<unsigned char> tab;
            tc_volume_tables(h, tab);
            e = cudaMalloc(&dtab, tab.size());
            if (e == cudaSuccess) e = cudaMemcpy(dtab, tab.data(), tab.size(), cudaMemcpyHostToDevice);
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(tc_volume_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, tcv::SMEM_BYTES);
            if (e != cudaSuccess) return e;
            tables[dev] = dtab;
        } else {
            dtab = it->second;
        }
    }
    cudaEvent_t e0, e1;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) return e;
    cudaEventRecord(e0, st);
    if (variant == 0) {
        const int64_t ncell = ntiles * tcv::M;
        cc_volume_kernel<<<(unsigned)((ncell + 255) / 256), 128, 0, st>>>(U, out, ncell);
    } else {
        int sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int64_t grid = std::min<int64_t>(ntiles, (int64_t)2 * (sms > 0 ? sms : 1));
        tc_volume_kernel<<<(unsigned)grid, 128, tcv::SMEM_BYTES, st>>>(U, out, dtab, ntiles, flag);
    }
    e = cudaGetLastError();
    cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess && ms) e = cudaEventElapsedTime(ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return e;
}
