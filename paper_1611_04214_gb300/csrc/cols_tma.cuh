// Column (y) sweeps in FP32 with tensor-memory-accelerator (TMA) tile loads and packed FP32x2
// arithmetic.  Same two-phase scan as the other column kernels (tile aggregates, carry scan down
// each column, tile results from the carries; Eq. IL / IR and the boundary correction of Sec. 3),
// laid out for sm_103a:
//   * a work item is one tile of R = 128 rows of a strip of 32 columns; one elected thread loads
//     the tile plus its stencil halo (R + M rows x 128 bytes per staged field) with one 2D
//     cp.async.bulk.tensor per field, completing on an mbarrier; 3 or 4 tiles are in flight;
//   * the two swept fields of a node (G(w) and w in pass 1, P and U in pass 3) share one 64-bit
//     register pair and every recurrence / stencil step is one fma.rn.f32x2;
//   * every mbarrier wait is bounded in time; a wait that runs out marks the block, the block
//     stops taking items, records the timeout in *status and returns.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include "sweep_common.cuh"

namespace molt {

// One 2D tensor map per staged field (at most two).
struct ColMaps {
    CUtensorMap m[2];
};

// ---- mbarrier / TMA primitives -----------------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(unsigned long long* b, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* b, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_test(unsigned long long* b, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// A tile copy completes in microseconds; one second without completion means it never will.
constexpr unsigned long long kWaitLimitNs = 1000000000ull;
__device__ __forceinline__ bool mbar_wait(unsigned long long* b, unsigned parity) {
    if (mbar_test(b, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_test(b, parity))
        if (global_ns() - t0 > kWaitLimitNs) return false;
    return true;
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// Status bit a kernel sets when one of its waits ran out of time.
constexpr unsigned kStatusWaitTimeout = 1u;

// Tiles in flight per block: 4 for one staged field, 3 for two (two blocks per SM either way).
__host__ __device__ constexpr int tma_col_stages(int ns) { return ns == 1 ? 4 : 3; }

// =========================================================================================
// The kernel.  Block = 8 warps; warp wy owns rows [wy*16, wy*16 + 16) of the tile, lane = column.
// Shared stage s holds, per staged field, rows r0 .. r0 + R + M - 1 (r0 = tile*R - M/2) of the
// strip; rows outside [0, n) arrive zero-filled and, on periodic lines, are read wrapped from
// global memory instead.  The buffer of item it-1 is refilled (item it+STAGES-1) right after the block
// barrier of item it, when no thread can still read it (STAGES = 3 or 4 tiles in flight).
// kFinal = false: tile aggregates; kFinal = true: tile results from the scan's carries.
// Requires nlines % 32 == 0 and n >= 256 (at least two tiles).
// =========================================================================================
template <int M, class Op, bool kFinal>
__global__ void __launch_bounds__(256, 2)
cols_tma_kernel(const __grid_constant__ LineParams<float> lp, const __grid_constant__ ColMaps maps,
                const __grid_constant__ PackedStencil pw, const Op op, int nlines, long long ld, int tiles,
                float* __restrict__ aggL, float* __restrict__ aggR, const float* __restrict__ carL,
                const float* __restrict__ carR, unsigned* status, unsigned long long* red_slots, int rev) {
    using T = float;
    constexpr int KY = 16, WY = 8, R = KY * WY, H = M / 2, ROWS = R + M;
    constexpr int NS = Op::NS, NF = Op::NF, NO = Op::NO, STAGES = tma_col_stages(Op::NS);
    constexpr unsigned kStageBytes = NS * ROWS * 32 * sizeof(float);
    using Ln = Lanes<NF>;
    using V = typename Ln::V;
    extern __shared__ __align__(128) unsigned char sm_tma[];
    // [STAGES][NS][ROWS][32], from the first 128-byte boundary (the launch adds 128 bytes)
    float* sm = reinterpret_cast<float*>(sm_tma + ((128u - (smem_u32(sm_tma) & 127u)) & 127u));
    __shared__ unsigned long long full[STAGES];
    __shared__ V sL[2][WY][32];
    __shared__ V sR[2][WY][32];

    const int lane = threadIdx.x & 31, wy = threadIdx.x >> 5;
    const int n = lp.n, N = lp.N, jb = lp.N - H + 1;
    const bool periodic = lp.bc == BC_PERIODIC;
    const T d = lp.d;
    const int nstrips = nlines >> 5;
    const int items = nstrips * tiles;
    T DK = T(1);
#pragma unroll
    for (int k = 0; k < KY - 1; ++k) DK *= d;
    const T DK1 = DK;   // d^{KY-1}
    DK *= d;            // d^{KY}
    const V dv = Ln::splat(d), DKv = Ln::splat(DK), nDKv = Ln::splat(-DK), nDK1v = Ln::splat(-DK1);
    auto WL = [&](int o) -> typename Ln::W {
        if constexpr (NF == 2) return pw.wl[o]; else return lp.wl[o];
    };
    auto WR = [&](int o) -> typename Ln::W {
        if constexpr (NF == 2) return pw.wr[o]; else return lp.wr[o];
    };
    // d^cnt of chunk i of a tile (cnt = rows of the chunk inside the line)
    auto chunk_decay = [&](int tile, int i) -> V {
        int c = n - (tile * R + i * KY);
        if (c >= KY) return DKv;
        T D = T(1);
        for (int k = 0; k < c; ++k) D *= d;
        return Ln::splat(D);
    };

    auto stage = [&](int s, int f) { return sm + (static_cast<size_t>(s) * NS + f) * ROWS * 32; };
    // rev = 1 takes the items from the last tile row up (the block order of the kernel that ran
    // before decides which end of the field is still in L2); results do not depend on it
    auto phys = [&](int itm) { return rev ? items - 1 - itm : itm; };
    auto issue = [&](int itm, int s) {
        const int strip = phys(itm) % nstrips, tile = phys(itm) / nstrips;
        mbar_expect_tx(&full[s], kStageBytes);
#pragma unroll
        for (int f = 0; f < NS; ++f) tma_load_2d(stage(s, f), &maps.m[f], strip * 32, tile * R - H, &full[s]);
    };

    if (threadIdx.x == 0) {
#pragma unroll
        for (int s = 0; s < STAGES; ++s) mbar_init(&full[s], 1);
        mbar_init_fence();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int j = 0; j < STAGES - 1; ++j)
            if (blockIdx.x + j * gridDim.x < items) issue(blockIdx.x + j * gridDim.x, j);
    }

    RedAcc<T> red{T(0), T(0)};
    bool failed = false;
    int it = 0;
    for (int item = blockIdx.x; item < items; item += gridDim.x, ++it) {
        const int s = it % STAGES;
        const int pb = it & 1;
        const bool arrived = mbar_wait(&full[s], static_cast<unsigned>((it / STAGES) & 1));

        const int strip = phys(item) % nstrips, tile = phys(item) / nstrips;
        const int line = strip * 32 + lane;
        const int r0 = tile * R - H;
        const int start = tile * R + wy * KY;
        int cnt = n - start;
        cnt = cnt < 0 ? 0 : (cnt > KY ? KY : cnt);
        const float* sb = stage(s, 0) + (wy * KY) * 32 + lane;
        const bool last = tile == tiles - 1;
        // final phase: the tile's carries, loaded first so that their latency hides behind the
        // window and the chunk aggregates
        T c0[NF], c1[NF];
#pragma unroll
        for (int q = 0; q < NF; ++q) {
            c0[q] = c1[q] = T(0);
            if constexpr (kFinal) {
                const size_t o = (static_cast<size_t>(q) * tiles + tile) * nlines + line;
                if (periodic || tile != 0) c0[q] = carL[o];
                if (periodic || !last) c1[q] = carR[o];
            }
        }

        // window of swept values: win[i] at position start - H + i (smem row wy*KY + i)
        V win[KY + M];
        const bool wrap = periodic && (start - H < 0 || start + KY + H > n);   // warp-uniform
        if (!wrap) {
#pragma unroll
            for (int i = 0; i < KY + M; ++i) {
                T sv[NS], fv[NF];
#pragma unroll
                for (int f = 0; f < NS; ++f) sv[f] = sb[static_cast<size_t>(f) * ROWS * 32 + i * 32];
                op.prologue(sv, fv);
                win[i] = Ln::make(fv);
            }
        } else {
#pragma unroll
            for (int i = 0; i < KY + M; ++i) {
                const int p = start - H + i;
                T sv[NS], fv[NF];
                if (p >= 0 && p < n) {
#pragma unroll
                    for (int f = 0; f < NS; ++f) sv[f] = sb[static_cast<size_t>(f) * ROWS * 32 + i * 32];
                } else {
                    const int q = p < 0 ? p + n : p - n;
#pragma unroll
                    for (int f = 0; f < NS; ++f) sv[f] = op.s[f][static_cast<long long>(q) * ld + line];
                }
                op.prologue(sv, fv);
                win[i] = Ln::make(fv);
            }
        }
        const bool interior = (cnt == KY) && (periodic || (start >= H && start + KY - 1 <= N - H));
        // wall values injected at the end nodes in the final phase (from the scan kernel)
        T injL[NF], injR[NF];
#pragma unroll
        for (int q = 0; q < NF; ++q) {
            injL[q] = injR[q] = T(0);
            if (kFinal && !periodic) {
                const size_t o = (static_cast<size_t>(q) * tiles + tile) * nlines + line;
                if (tile == 0) injL[q] = carL[o];
                if (tile == tiles - 1) injR[q] = carR[o];
            }
        }
        // all NF swept values at line position p (prologue applied), from the stage or from global
        // memory when p lies outside it
        auto at_v = [&](int p) -> V {
            const int rr = p - r0;
            T sv[NS], fv[NF];
            if (rr >= 0 && rr < ROWS) {
#pragma unroll
                for (int f = 0; f < NS; ++f) sv[f] = stage(s, f)[rr * 32 + lane];
            } else {
#pragma unroll
                for (int f = 0; f < NS; ++f) sv[f] = op.s[f][static_cast<long long>(p) * ld + line];
            }
            op.prologue(sv, fv);
            return Ln::make(fv);
        };
        // J^L, J^R at chunk position k of a chunk that is not interior (it touches a wall of a
        // non-periodic line, or it is the ragged end of the line): interior positions from the
        // window; the first and last H positions of a non-periodic line from the shifted wall
        // stencils (Sec. 3.2 reading) on wall nodes 0..M or N-M..N, whose prologue is evaluated
        // once per node into wv; zero past the end of the line.  In the final phase J^L_0 = B_a and
        // J^R_N = B_b (injected, from the scan).  Same operations in the same order as
        // local_integrals.  (A chunk of 16 rows touches at most one wall: lines have n >= 256.)
        const bool nearA = !periodic && start < H;
        const bool nearB = !periodic && start + cnt - 1 >= jb;
        V wv[M + 1];
        if (!interior) {
            const int base = nearA ? 0 : N - M;
#pragma unroll
            for (int o = 0; o <= M; ++o) wv[o] = (nearA || nearB) ? at_v(base + o) : Ln::zero();
        }
        auto jl_e = [&](int k) -> V {
            const int j = start + k;
            V a = Ln::zero();
            if (nearA && j < H) {
                if (j == 0) return Ln::make(injL);
                a = Ln::fma(Ln::splat(lp.wlA[j - 1][0]), wv[0], a);
#pragma unroll
                for (int o = 1; o <= M; ++o) a = Ln::fma(Ln::splat(lp.wlA[j - 1][o]), wv[o], a);
            } else if (nearB && j >= jb) {
                a = Ln::fma(Ln::splat(lp.wlB[j - jb][0]), wv[0], a);
#pragma unroll
                for (int o = 1; o <= M; ++o) a = Ln::fma(Ln::splat(lp.wlB[j - jb][o]), wv[o], a);
            } else {
                a = Ln::fma(WL(0), win[k], a);
#pragma unroll
                for (int o = 1; o <= M; ++o) a = Ln::fma(WL(o), win[k + o], a);
            }
            return a;
        };
        auto jr_e = [&](int k) -> V {
            const int j = start + k;
            V a = Ln::zero();
            if (nearA && j < H) {
                a = Ln::fma(Ln::splat(lp.wrA[j][0]), wv[0], a);
#pragma unroll
                for (int o = 1; o <= M; ++o) a = Ln::fma(Ln::splat(lp.wrA[j][o]), wv[o], a);
            } else if (nearB && j >= jb) {
                if (j == N) return Ln::make(injR);
                a = Ln::fma(Ln::splat(lp.wrB[j - jb][0]), wv[0], a);
#pragma unroll
                for (int o = 1; o <= M; ++o) a = Ln::fma(Ln::splat(lp.wrB[j - jb][o]), wv[o], a);
            } else {
                a = Ln::fma(WR(0), win[k], a);
#pragma unroll
                for (int o = 1; o <= M; ++o) a = Ln::fma(WR(o), win[k + o], a);
            }
            return a;
        };

        // ---- chunk aggregates (shifted recurrences, see cols_pipe_kernel) ----
        V aL, aR;
        if (interior) {
            V S = Ln::zero();
#pragma unroll
            for (int k = 0; k < KY; ++k) S = Ln::fma(dv, S, win[k]);
            V a = Ln::fma(WL(0), S, Ln::zero());
#pragma unroll
            for (int o = 0; o < M; ++o) {
                S = Ln::fma(dv, S, Ln::fma(nDKv, win[o], win[KY + o]));
                a = Ln::fma(WL(o + 1), S, a);
            }
            V Rr = Ln::zero();
#pragma unroll
            for (int k = KY - 1; k >= 0; --k) Rr = Ln::fma(dv, Rr, win[k + M]);
            V b = Ln::fma(WR(M), Rr, Ln::zero());
#pragma unroll
            for (int o = M - 1; o >= 0; --o) {
                Rr = Ln::fma(dv, Ln::fma(nDK1v, win[KY + o], Rr), win[o]);
                b = Ln::fma(WR(o), Rr, b);
            }
            aL = a;
            aR = b;
        } else {
            V a = Ln::zero(), b = Ln::zero();
#pragma unroll
            for (int k = 0; k < KY; ++k)
                if (k < cnt) a = Ln::fma(dv, a, jl_e(k));
#pragma unroll
            for (int k = KY - 1; k >= 0; --k)
                if (k < cnt) b = Ln::fma(dv, b, jr_e(k));
            aL = a;
            aR = b;
        }
        sL[pb][wy][lane] = aL;
        sR[pb][wy][lane] = aR;
        // every thread is done with the stage of item it-1: refill it; agree on timeouts
        failed = __syncthreads_or(!arrived) != 0;
        if (failed) break;
        if (threadIdx.x == 0 && item + (STAGES - 1) * gridDim.x < items)
            issue(item + (STAGES - 1) * gridDim.x, (it + STAGES - 1) % STAGES);

        if constexpr (!kFinal) {
            if (wy == 0) {
                V a = Ln::zero(), b = Ln::zero();
                if (!last) {
#pragma unroll
                    for (int i = 0; i < WY; ++i) a = Ln::fma(a, DKv, sL[pb][i][lane]);
#pragma unroll
                    for (int i = WY - 1; i >= 0; --i) b = Ln::fma(b, DKv, sR[pb][i][lane]);
                } else {
                    for (int i = 0; i < WY; ++i) a = Ln::fma(a, chunk_decay(tile, i), sL[pb][i][lane]);
                    for (int i = WY - 1; i >= 0; --i) b = Ln::fma(b, chunk_decay(tile, i), sR[pb][i][lane]);
                }
#pragma unroll
                for (int q = 0; q < NF; ++q) {
                    const size_t o = (static_cast<size_t>(q) * tiles + tile) * nlines + line;
                    aggL[o] = Ln::get(a, q);
                    aggR[o] = Ln::get(b, q);
                }
            }
        } else {
            V cl = Ln::make(c0), cr = Ln::make(c1);
            if (!last) {
                for (int i = 0; i < wy; ++i) cl = Ln::fma(cl, DKv, sL[pb][i][lane]);
                for (int i = WY - 1; i > wy; --i) cr = Ln::fma(cr, DKv, sR[pb][i][lane]);
            } else {
                for (int i = 0; i < wy; ++i) cl = Ln::fma(cl, chunk_decay(tile, i), sL[pb][i][lane]);
                for (int i = WY - 1; i > wy; --i) cr = Ln::fma(cr, chunk_decay(tile, i), sR[pb][i][lane]);
            }
            // P^R backward from the right carry, then P^L forward added (Eq. IL / IR)
            V out[KY];
            if (interior) {
                V p = cr;
#pragma unroll
                for (int k = KY - 1; k >= 0; --k) {
                    V a = Ln::fma(WR(0), win[k], Ln::zero());
#pragma unroll
                    for (int o = 1; o <= M; ++o) a = Ln::fma(WR(o), win[k + o], a);
                    p = Ln::fma(dv, p, a);
                    out[k] = p;
                }
                V s2 = cl;
#pragma unroll
                for (int k = 0; k < KY; ++k) {
                    V a = Ln::fma(WL(0), win[k], Ln::zero());
#pragma unroll
                    for (int o = 1; o <= M; ++o) a = Ln::fma(WL(o), win[k + o], a);
                    s2 = Ln::fma(dv, s2, a);
                    out[k] = Ln::add(out[k], s2);
                }
            } else {
                V p = cr;
#pragma unroll
                for (int k = KY - 1; k >= 0; --k) {
                    out[k] = Ln::zero();
                    if (k < cnt) {
                        p = Ln::fma(dv, p, jr_e(k));
                        out[k] = p;
                    }
                }
                V s2 = cl;
#pragma unroll
                for (int k = 0; k < KY; ++k)
                    if (k < cnt) {
                        s2 = Ln::fma(dv, s2, jl_e(k));
                        out[k] = Ln::add(out[k], s2);
                    }
            }
            T* ob[NO];
#pragma unroll
            for (int o = 0; o < NO; ++o) ob[o] = op.o[o] + static_cast<long long>(start) * ld + line;
            auto emit = [&](int k) {
                T h[NF], sv[NS], av[1] = {T(0)}, ov[NO];
#pragma unroll
                for (int q = 0; q < NF; ++q) h[q] = Ln::get(out[k], q);
#pragma unroll
                for (int f = 0; f < NS; ++f) sv[f] = sb[static_cast<size_t>(f) * ROWS * 32 + (k + H) * 32];
                op.epilogue(h, sv, av, ov, red);
#pragma unroll
                for (int o = 0; o < NO; ++o) ob[o][static_cast<long long>(k) * ld] = ov[o];
            };
            if (cnt == KY) {
#pragma unroll
                for (int k = 0; k < KY; ++k) emit(k);
            } else {
#pragma unroll
                for (int k = 0; k < KY; ++k)
                    if (k < cnt) emit(k);
            }
        }
    }
    if (failed) {
        // stop here; let the copies this block still has in flight (items it .. it+STAGES-2,
        // those that were issued) land, each wait bounded, before exiting
        if (threadIdx.x == 0) {
            for (int j = 0; j <= STAGES - 2; ++j) {
                const int itm = blockIdx.x + (it + j) * gridDim.x;
                if (itm < items) mbar_wait(&full[(it + j) % STAGES], static_cast<unsigned>(((it + j) / STAGES) & 1));
            }
            if (status) atomicOr(status, kStatusWaitTimeout);
        }
        return;
    }
    if (Op::kReduce) block_reduce_store<T>(red, red_slots);
}

}  // namespace molt
