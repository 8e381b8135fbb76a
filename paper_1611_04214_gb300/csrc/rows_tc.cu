// Row (x) sweeps of H_c on periodic lines as tensor-core products: the chunked form of the
// recurrences of Eq. IL / IR on the 5th-generation tensor cores (tcgen05), an experiment on the
// FP16 split-precision variant of the line sweep.
//
// A line is cut into chunks of C = 128 nodes.  Inside a chunk both recurrences started from zero
// are linear in the chunk's window of C + M node values (the chunk and M/2 halo nodes on each
// side, Sec. 3.2 local quadrature folded in):
//   I^L_local = T_L W_L v,  (T_L)_{ij} = d^{i-j} (i >= j),  (W_L v)_m = J^L at chunk node m,
//   I^R_local = T_R W_R v,  (T_R)_{ij} = d^{j-i} (i <= j),  (W_R v)_m = J^R at chunk node m,
// so A_L = T_L W_L and A_R = T_R W_R are 128 x (C + M) matrices, the same for every chunk of every
// line, and one product D = A V with one column of V per chunk computes the local parts of a whole
// tile of chunks.  The carries between chunks (the last row of A_L v, the first row of A_R v) are
// scanned down each line in FP32 with the periodic boundary correction (Eq. homogeneous) in FP64,
// and each output is out_i = D_L[i] + d^{i+1} carry_L + D_R[i] + d^{C-i} carry_R.
//
// Precision: A and V are split into FP16 high and low parts (x = hi + lo, lo = fp16(x - hi)) and
// D = A_hi V_hi + A_hi V_lo + A_lo V_hi, accumulated in FP32 in tensor memory: about 22 bits of
// each operand, the A_lo V_lo term below FP32 rounding.
//
// Layout: operands in shared memory in the K-major canonical layout without swizzle (8 x 8 FP16
// core matrices of 128 bytes; 128 bytes between core matrices along K, 2304 bytes between groups
// of 8 rows); D_L and D_R in 128 tensor-memory columns; one elected thread issues the MMAs and
// commits them to an mbarrier whose wait is bounded in time.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "cols_tma.cuh"
#include "molt_internal.h"

namespace molt {
namespace tc {

constexpr int C = 128;                  // nodes per chunk = rows of the product (M of the MMA)
constexpr int KP = 144;                 // chunk window C + M (M <= 6) padded to a multiple of 16
constexpr int NT = 64;                  // chunks per tile (N of the MMA)
constexpr int KSTEPS = KP / 16;         // MMAs of K = 16 per product
constexpr int CORE = 128;               // bytes of one 8 x 8 FP16 core matrix
constexpr int SBO = (KP / 8) * CORE;    // bytes between groups of 8 rows
constexpr int MAT_A = (C / 8) * SBO;    // bytes of one 128 x 144 FP16 operand
constexpr int MAT_B = (NT / 8) * SBO;   // bytes of one 64 x 144 FP16 operand
constexpr int THREADS = 128;
constexpr int TMEM_COLS = 128;          // D_L: columns 0..63, D_R: 64..127
constexpr int SMEM = 4 * MAT_A + 2 * MAT_B + 8192 + 1024;   // operands, slack, alignment
// F32 accumulator, FP16 A and B, both K-major, N = 64, M = 128
constexpr unsigned IDESC = (1u << 4) | ((NT >> 3) << 17) | ((C >> 4) << 24);

// byte offset of element (row r, column k) of a K-major operand
__host__ __device__ constexpr int core_offset(int r, int k) {
    return (r >> 3) * SBO + (k >> 3) * CORE + (r & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ unsigned long long desc(unsigned addr) {
    unsigned long long d = static_cast<unsigned long long>((addr >> 4) & 0x3FFFu);   // start address
    d |= static_cast<unsigned long long>((CORE >> 4) & 0x3FFF) << 16;                // next core matrix along K
    d |= static_cast<unsigned long long>((SBO >> 4) & 0x3FFF) << 32;                 // next 8 rows
    d |= 1ull << 46;                                                                 // descriptor version
    return d;                                                                        // no swizzle
}

__device__ __forceinline__ void mma(unsigned d_tmem, unsigned long long a, unsigned long long b, unsigned acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(d_tmem), "l"(a), "l"(b), "r"(IDESC), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void commit(unsigned long long* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void ld16(unsigned taddr, float* v) {
    unsigned r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// FP64 operands A_L, A_R ([2][C][KP], row-major) -> FP16 high / low parts in the core layout:
// [A_L hi][A_L lo][A_R hi][A_R lo].
__global__ void pack_kernel(const double* a, unsigned char* packed) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 2 * C * KP) return;
    const int m = idx / (C * KP), r = (idx / KP) % C, k = idx % KP;
    const double x = a[idx];
    const __half hi = __double2half(x);
    const __half lo = __double2half(x - static_cast<double>(__half2float(hi)));
    unsigned char* base = packed + static_cast<size_t>(2 * m) * MAT_A;
    *reinterpret_cast<__half*>(base + core_offset(r, k)) = hi;
    *reinterpret_cast<__half*>(base + MAT_A + core_offset(r, k)) = lo;
}

template <int M>
__global__ void __launch_bounds__(THREADS, 1)
rows_kernel(const float* __restrict__ in, float* __restrict__ out, int n, int nlines,
            const unsigned char* __restrict__ packed, float nu, double inv1mmu, unsigned* status) {
    constexpr int H = M / 2;
    extern __shared__ unsigned char tc_smem_raw[];
    unsigned char* sm = tc_smem_raw + ((1024u - (smem_u32(tc_smem_raw) & 1023u)) & 1023u);
    unsigned char* sA = sm;                  // A_L hi, A_L lo, A_R hi, A_R lo
    unsigned char* sB = sm + 4 * MAT_A;      // V hi, V lo
    __shared__ unsigned long long mbar;
    __shared__ unsigned tmem_holder;
    __shared__ float s_aggL[NT], s_aggR[NT], s_carL[NT], s_carR[NT];

    const int tid = threadIdx.x, warp = tid >> 5;
    // operands A into shared memory once; V is rebuilt per tile
    for (int i = tid; i < 4 * MAT_A / 16; i += THREADS)
        reinterpret_cast<uint4*>(sA)[i] = reinterpret_cast<const uint4*>(packed)[i];
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_holder)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(&mbar, 1);
        mbar_init_fence();
    }
    fence_proxy();
    fence_before();
    __syncthreads();
    fence_after();
    const unsigned tmem = tmem_holder;
    const unsigned aaddr = smem_u32(sA), baddr = smem_u32(sB);

    const int cpl = n / C;                           // chunks per line (divides NT)
    const long long tiles = static_cast<long long>(nlines) * cpl / NT;
    const float DC = expf(-nu * static_cast<float>(C));
    const float pwl = expf(-nu * static_cast<float>(tid + 1));   // d^{i+1}, i = this thread's row
    const float pwr = expf(-nu * static_cast<float>(C - tid));   // d^{C-i}
    bool failed = false;
    int it = 0;
    for (long long tl = blockIdx.x; tl < tiles; tl += gridDim.x, ++it) {
        // ---- V: chunk c = tid % 64, window half tid / 64 (72 of the 144 window entries) ----
        {
            const int c = tid & (NT - 1), half = tid >> 6;
            const long long gc = tl * NT + c;
            const long long line = gc / cpl;
            const int start = static_cast<int>(gc % cpl) * C;
            const float* row = in + line * n;
#pragma unroll
            for (int kb = 0; kb < KP / 16; ++kb) {
                const int kb8 = half * (KP / 16) + kb;   // core column of 8 window entries
                unsigned hw[4], lw[4];
#pragma unroll
                for (int e = 0; e < 8; e += 2) {
                    unsigned short hs[2], ls[2];
#pragma unroll
                    for (int q = 0; q < 2; ++q) {
                        const int k = kb8 * 8 + e + q;
                        float v = 0.0f;
                        if (k < C + M) {
                            int p = start - H + k;
                            p = p < 0 ? p + n : (p >= n ? p - n : p);
                            v = __ldg(row + p);
                        }
                        const __half h = __float2half_rn(v);
                        hs[q] = __half_as_ushort(h);
                        ls[q] = __half_as_ushort(__float2half_rn(v - __half2float(h)));
                    }
                    hw[e / 2] = static_cast<unsigned>(hs[0]) | (static_cast<unsigned>(hs[1]) << 16);
                    lw[e / 2] = static_cast<unsigned>(ls[0]) | (static_cast<unsigned>(ls[1]) << 16);
                }
                const int off = core_offset(c, kb8 * 8);
                *reinterpret_cast<uint4*>(sB + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                *reinterpret_cast<uint4*>(sB + MAT_B + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
            }
        }
        fence_proxy();        // the generic-proxy writes of V are visible to the tensor cores
        fence_before();
        __syncthreads();      // ... and every thread's TMEM reads of the previous tile are done
        fence_after();
        // ---- D_L = A_L V, D_R = A_R V as three FP16 products each ----
        if (tid == 0) {
#pragma unroll
            for (int side = 0; side < 2; ++side) {
                const unsigned d = tmem + side * NT;
                const unsigned abase = aaddr + side * 2 * MAT_A;
#pragma unroll
                for (int prod = 0; prod < 3; ++prod) {
                    const unsigned a0 = abase + (prod == 2 ? MAT_A : 0);   // hi, hi, lo
                    const unsigned b0 = baddr + (prod == 1 ? MAT_B : 0);   // hi, lo, hi
#pragma unroll
                    for (int s = 0; s < KSTEPS; ++s)
                        mma(d, desc(a0 + s * 2 * CORE), desc(b0 + s * 2 * CORE), (prod | s) != 0 ? 1u : 0u);
                }
            }
            commit(&mbar);
        }
        const bool done = mbar_wait(&mbar, static_cast<unsigned>(it & 1));
        failed = __syncthreads_or(!done) != 0;
        if (failed) break;
        fence_after();
        // ---- D rows of this thread (row = tid) ----
        float DL[NT], DR[NT];
        const unsigned trow = tmem + (static_cast<unsigned>(warp * 32) << 16);
#pragma unroll
        for (int j = 0; j < NT / 16; ++j) {
            ld16(trow + j * 16, DL + j * 16);
            ld16(trow + NT + j * 16, DR + j * 16);
        }
        ld_wait();
        // ---- carries: chunk aggregates (last row of D_L, first of D_R) scanned down each line ----
        if (tid == C - 1) {
#pragma unroll
            for (int c = 0; c < NT; ++c) s_aggL[c] = DL[c];
        }
        if (tid == 0) {
#pragma unroll
            for (int c = 0; c < NT; ++c) s_aggR[c] = DR[c];
        }
        __syncthreads();
        const int lpt = NT / cpl;                    // lines in the tile
        if (tid < 2 * lpt) {
            const int base = (tid >> 1) * cpl;
            float E = 0.0f;
            if ((tid & 1) == 0) {
                for (int c = 0; c < cpl; ++c) {
                    s_carL[base + c] = E;
                    E = fmaf(E, DC, s_aggL[base + c]);
                }
                const float X = static_cast<float>(static_cast<double>(E) * inv1mmu);   // periodic B_a
                for (int c = 0; c < cpl; ++c) s_carL[base + c] = fmaf(expf(-nu * static_cast<float>(c * C)), X, s_carL[base + c]);
            } else {
                for (int c = cpl - 1; c >= 0; --c) {
                    s_carR[base + c] = E;
                    E = fmaf(E, DC, s_aggR[base + c]);
                }
                const float X = static_cast<float>(static_cast<double>(E) * inv1mmu);   // periodic B_b
                for (int c = 0; c < cpl; ++c)
                    s_carR[base + c] = fmaf(expf(-nu * static_cast<float>(n - c * C - C)), X, s_carR[base + c]);
            }
        }
        __syncthreads();
        // ---- outputs: node tid of every chunk of the tile (a warp stores 32 consecutive nodes) ----
#pragma unroll
        for (int c = 0; c < NT; ++c) {
            const long long gc = tl * NT + c;
            const long long line = gc / cpl;
            const int pos = static_cast<int>(gc % cpl) * C + tid;
            out[line * n + pos] = fmaf(pwr, s_carR[c], fmaf(pwl, s_carL[c], DL[c] + DR[c]));
        }
        fence_before();
    }
    if (failed && tid == 0) {
        mbar_wait(&mbar, static_cast<unsigned>(it & 1));   // bounded: let the products in flight finish
        if (status) atomicOr(status, kStatusWaitTimeout);
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}

template <int M>
cudaError_t launch(const LineParams<double>& lp, const unsigned char* packed, const float* in, float* out, int nlines,
                   unsigned* status, cudaStream_t st) {
    static const cudaError_t optin =
        cudaFuncSetAttribute(rows_kernel<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
    if (optin != cudaSuccess) return optin;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long tiles = static_cast<long long>(nlines) * (lp.n / C) / NT;
    const int grid = static_cast<int>(tiles < sms ? tiles : sms);
    rows_kernel<M><<<grid, THREADS, SMEM, st>>>(in, out, lp.n, nlines, packed, static_cast<float>(lp.nu), lp.inv1mmu,
                                                status);
    return cudaGetLastError();
}

}  // namespace tc

size_t rows_tc_workspace_bytes() { return 2 * sizeof(double) * tc::C * tc::KP + 4 * static_cast<size_t>(tc::MAT_A); }

bool rows_tc_supported(int n, int nlines, int M) {
    if (M > 6 || n < 1024 || n > 8192 || (n & (n - 1)) != 0) return false;
    const int cpl = n / tc::C;
    return (static_cast<long long>(nlines) * cpl) % tc::NT == 0;
}

// Host: the FP64 operands A_L = T_L W_L and A_R = T_R W_R of one periodic line inverse; window
// entry k of a chunk is node (chunk start - M/2 + k), entries k >= C + M are zero.
static void build_operands(const LineParams<double>& lp, std::vector<double>& a) {
    using namespace tc;
    a.assign(2 * C * KP, 0.0);
    std::vector<double> pw(C);
    pw[0] = 1.0;
    for (int i = 1; i < C; ++i) pw[i] = pw[i - 1] * lp.d;
    for (int i = 0; i < C; ++i) {
        for (int m = 0; m <= i; ++m)           // J^L at chunk node m reaches row i with d^{i-m}
            for (int o = 0; o <= lp.M; ++o) a[static_cast<size_t>(i) * KP + m + o] += pw[i - m] * lp.wl[o];
        for (int m = i; m < C; ++m)            // J^R at chunk node m reaches row i with d^{m-i}
            for (int o = 0; o <= lp.M; ++o) a[static_cast<size_t>(C + i) * KP + m + o] += pw[m - i] * lp.wr[o];
    }
}

cudaError_t rows_tc_prepare(const LineParams<double>& lp, void* workspace, cudaStream_t st) {
    std::vector<double> a;
    build_operands(lp, a);
    double* staged = static_cast<double*>(workspace);
    unsigned char* packed = static_cast<unsigned char*>(workspace) + 2 * sizeof(double) * tc::C * tc::KP;
    cudaError_t e = cudaMemcpyAsync(staged, a.data(), a.size() * sizeof(double), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(packed, 0, 4 * static_cast<size_t>(tc::MAT_A), st);
    if (e != cudaSuccess) return e;
    tc::pack_kernel<<<(2 * tc::C * tc::KP + 255) / 256, 256, 0, st>>>(staged, packed);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(st);   // the host vector is released on return
}

cudaError_t rows_tc(const LineParams<double>& lp, const void* workspace, const float* in, float* out, int nlines,
                    unsigned* status, cudaStream_t st) {
    if (lp.bc != BC_PERIODIC || !rows_tc_supported(lp.n, nlines, lp.M)) return cudaErrorInvalidValue;
    const unsigned char* packed = static_cast<const unsigned char*>(workspace) + 2 * sizeof(double) * tc::C * tc::KP;
    // the kernels of the three orders share one function type, so each opts in through its own
    // function-local static
    switch (lp.M) {
        case 2: return tc::launch<2>(lp, packed, in, out, nlines, status, st);
        case 4: return tc::launch<4>(lp, packed, in, out, nlines, status, st);
        default: return tc::launch<6>(lp, packed, in, out, nlines, status, st);
    }
}

}  // namespace molt
