// Line-sweep kernels of H_c (Sec. 3.2) along contiguous rows and along strided columns.
#pragma once

#include "sweep_common.cuh"

namespace molt {

// =========================================================================================
// Rows: each line is staged once in shared memory (coalesced, prologue applied), a team of
// TL = 2^tl_log2 threads owns it (K positions per thread), and the result goes back through
// shared memory to coalesced stores (epilogue applied).  One read and one write per element.
// Shared layout: [line in block][field][position + position/32] (the pad keeps the chunked
// per-thread reads free of bank conflicts).
// =========================================================================================
// Body of one block: lines line0 .. line0 + lpb - 1 of nlines; sm = the block's dynamic shared
// memory (lpb * NF * pitch values).  Shared by rows_kernel and the batched row kernel.
template <typename T, int M, int K, class Op>
__device__ __forceinline__ void rows_body(const LineParams<T>& lp, const Op& op, int nlines, int tl_log2, int lpb,
                                          int pitch, int line0, T* sm, unsigned long long* red_slots) {
    constexpr int NF = Op::NF;
    constexpr int H = M / 2;
    __shared__ T s_scan[32][2 + 2 * NF];   // per-warp segments: D_f, D_b, A_f[NF], A_b[NF]
    __shared__ T s_tot[32][2 * NF];        // per-line totals (lines spanning several warps)
    __shared__ T s_bnd[128][2 * NF];       // per-line carries / B values from the FP64 solve

    const int n = lp.n;
    const bool periodic = lp.bc == BC_PERIODIC;
    const int TL = 1 << tl_log2;
    const int tid = threadIdx.x;
    const int lib = tid >> tl_log2;
    const int t = tid & (TL - 1);

    // ---- stage the block's lines (prologue): batches of U independent loads per thread ----
    constexpr int U = 8;
    for (int l = 0; l < lpb; ++l) {
        const int gl = line0 + l;
        if (gl >= nlines) break;
        T* dst = sm + static_cast<size_t>(l) * NF * pitch;
        for (int base = 0; base < n; base += U * blockDim.x) {
            T f[U][NF];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int p = base + u * blockDim.x + tid;
                if (p < n) op.load(gl, p, f[u]);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int p = base + u * blockDim.x + tid;
                if (p < n) {
#pragma unroll
                    for (int q = 0; q < NF; ++q) dst[q * pitch + p + (p >> 5)] = f[u][q];
                }
            }
        }
    }
    __syncthreads();

    const bool in_block = lib < lpb;            // a 32-thread minimum block may exceed lpb lines
    const int line = line0 + lib;
    const int start = t * K;
    int cnt = n - start;
    cnt = cnt < 0 ? 0 : (cnt > K ? K : cnt);
    if (!in_block || line >= nlines) cnt = 0;
    const T d = lp.d;
    const T* base = sm + static_cast<size_t>(in_block ? lib : 0) * NF * pitch;

    T JL[NF][K], JR[NF][K];
    T aL[NF], aR[NF];
#pragma unroll
    for (int q = 0; q < NF; ++q) {
        const T* fb = base + q * pitch;
        if (cnt > 0) {
            T win[K + M];
#pragma unroll
            for (int i = 0; i < K + M; ++i) {
                const int p = fold_pos(start - H + i, n, periodic);
                win[i] = fb[p + (p >> 5)];
            }
            local_integrals<T, M, K>(lp, start, cnt, win, [&](int p) { return fb[p + (p >> 5)]; }, JL[q], JR[q]);
        } else {
#pragma unroll
            for (int k = 0; k < K; ++k) JL[q][k] = JR[q][k] = T(0);
        }
        chunk_aggregates<T, K>(d, cnt, JL[q], JR[q], aL[q], aR[q]);
    }
    T D = T(1);
#pragma unroll
    for (int k = 0; k < K; ++k)
        if (k < cnt) D *= d;

    // ---- scan the chunk segments over the TL threads of the line ----
    const int lane = tid & 31;
    const int w = TL < 32 ? TL : 32;
    const int li = lane & (w - 1);
    T Df = D, Db = D, Af[NF], Ab[NF];
#pragma unroll
    for (int q = 0; q < NF; ++q) {
        Af[q] = aL[q];
        Ab[q] = aR[q];
    }
    for (int o = 1; o < w; o <<= 1) {
        const T dpf = __shfl_up_sync(kFull, Df, o, w);
        const T dpb = __shfl_down_sync(kFull, Db, o, w);
#pragma unroll
        for (int q = 0; q < NF; ++q) {
            const T apf = __shfl_up_sync(kFull, Af[q], o, w);
            const T apb = __shfl_down_sync(kFull, Ab[q], o, w);
            if (li >= o) Af[q] = fma(apf, Df, Af[q]);
            if (li + o < w) Ab[q] = fma(apb, Db, Ab[q]);
        }
        if (li >= o) Df = dpf * Df;
        if (li + o < w) Db = dpb * Db;
    }
    // exclusive values (segment entering this chunk), totals of the line
    T Dxf = __shfl_up_sync(kFull, Df, 1, w), Dxb = __shfl_down_sync(kFull, Db, 1, w);
    T Axf[NF], Axb[NF], TotF[NF], TotB[NF];
#pragma unroll
    for (int q = 0; q < NF; ++q) {
        Axf[q] = __shfl_up_sync(kFull, Af[q], 1, w);
        Axb[q] = __shfl_down_sync(kFull, Ab[q], 1, w);
        TotF[q] = __shfl_sync(kFull, Af[q], w - 1, w);
        TotB[q] = __shfl_sync(kFull, Ab[q], 0, w);
        if (li == 0) Axf[q] = T(0);
        if (li == w - 1) Axb[q] = T(0);
    }
    if (li == 0) Dxf = T(1);
    if (li == w - 1) Dxb = T(1);
    if (TL > 32) {
        // Lines span wpl = TL/32 warps: the first warp of each line scans the warp totals
        // (log depth) and leaves each warp the segment entering it.
        const int warp = tid >> 5;
        const int wpl = TL >> 5;
        const int first = (warp / wpl) * wpl;
        if (lane == 31) {
            s_scan[warp][0] = Df;
#pragma unroll
            for (int q = 0; q < NF; ++q) s_scan[warp][2 + q] = Af[q];
        }
        if (lane == 0) {
            s_scan[warp][1] = Db;
#pragma unroll
            for (int q = 0; q < NF; ++q) s_scan[warp][2 + NF + q] = Ab[q];
        }
        __syncthreads();
        if (warp == first) {
            const bool has = lane < wpl;
            T fD = has ? s_scan[first + lane][0] : T(1);
            T bD = has ? s_scan[first + lane][1] : T(1);
            T fA[NF], bA[NF];
#pragma unroll
            for (int q = 0; q < NF; ++q) {
                fA[q] = has ? s_scan[first + lane][2 + q] : T(0);
                bA[q] = has ? s_scan[first + lane][2 + NF + q] : T(0);
            }
            for (int o = 1; o < 32; o <<= 1) {
                const T pfD = __shfl_up_sync(kFull, fD, o);
                const T pbD = __shfl_down_sync(kFull, bD, o);
#pragma unroll
                for (int q = 0; q < NF; ++q) {
                    const T pf = __shfl_up_sync(kFull, fA[q], o);
                    const T pb = __shfl_down_sync(kFull, bA[q], o);
                    if (lane >= o) fA[q] = fma(pf, fD, fA[q]);
                    if (lane + o < 32) bA[q] = fma(pb, bD, bA[q]);
                }
                if (lane >= o) fD = pfD * fD;
                if (lane + o < 32) bD = pbD * bD;
            }
            T exF[NF], exB[NF], totF[NF], totB[NF];
#pragma unroll
            for (int q = 0; q < NF; ++q) {
                exF[q] = __shfl_up_sync(kFull, fA[q], 1);
                exB[q] = __shfl_down_sync(kFull, bA[q], 1);
                totF[q] = __shfl_sync(kFull, fA[q], 31);
                totB[q] = __shfl_sync(kFull, bA[q], 0);
                if (lane == 0) exF[q] = T(0);
                if (lane == 31 || lane + 1 >= wpl) exB[q] = T(0);
            }
            __syncwarp();
            if (has) {
#pragma unroll
                for (int q = 0; q < NF; ++q) {
                    s_scan[first + lane][2 + q] = exF[q];          // forward segment entering warp
                    s_scan[first + lane][2 + NF + q] = exB[q];     // backward segment entering warp
                    if (lane == 0) {
                        s_tot[first / wpl][q] = totF[q];
                        s_tot[first / wpl][NF + q] = totB[q];
                    }
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < NF; ++q) {
            Axf[q] = fma(s_scan[warp][2 + q], Dxf, Axf[q]);
            Axb[q] = fma(s_scan[warp][2 + NF + q], Dxb, Axb[q]);
            TotF[q] = s_tot[first / wpl][q];
            TotB[q] = s_tot[first / wpl][NF + q];
        }
    }

    // ---- boundary correction: one FP64 2x2 solve per line, then carries in T ----
    if (t == 0 && in_block) {
#pragma unroll
        for (int q = 0; q < NF; ++q) {
            const double I0 = static_cast<double>(TotB[q]);
            const double IN = static_cast<double>(TotF[q]);
            double xl, xr;
            if (periodic) {
                xl = IN * lp.inv1mmu;                 // carry entering position 0
                xr = I0 * lp.inv1mmu;                 // carry entering position n-1
            } else {
                xl = lp.bAA * I0 + lp.bAB * IN;       // B_a
                xr = lp.bBA * I0 + lp.bBB * IN;       // B_b
            }
            s_bnd[lib][q] = static_cast<T>(xl);
            s_bnd[lib][NF + q] = static_cast<T>(xr);
        }
    }
    __syncthreads();
    const int end = start + cnt - 1;
    T cL[NF], cR[NF];
    if (cnt > 0) {
        const T pl = dev_exp(-lp.nu * T(periodic ? start : start - 1));
        const T pr = dev_exp(-lp.nu * T(periodic ? n - start - cnt : n - start - cnt - 1));
#pragma unroll
        for (int q = 0; q < NF; ++q) {
            const T xl = s_bnd[lib][q], xr = s_bnd[lib][NF + q];
            if (periodic) {
                cL[q] = fma(pl, xl, Axf[q]);
                cR[q] = fma(pr, xr, Axb[q]);
            } else {
                if (start == 0) {
                    JL[q][0] += xl;                   // P^L_0 = B_a
                    cL[q] = T(0);
                } else {
                    cL[q] = fma(pl, xl, Axf[q]);
                }
                if (end == n - 1) {
#pragma unroll
                    for (int k = 0; k < K; ++k)
                        if (k == cnt - 1) JR[q][k] += xr;   // P^R_N = B_b
                    cR[q] = T(0);
                } else {
                    cR[q] = fma(pr, xr, Axb[q]);
                }
            }
        }
    } else {
#pragma unroll
        for (int q = 0; q < NF; ++q) cL[q] = cR[q] = T(0);
    }
#pragma unroll
    for (int q = 0; q < NF; ++q) chunk_finish<T, K>(d, cnt, cL[q], cR[q], JL[q], JR[q]);

    // ---- results back through shared memory, then coalesced epilogue ----
    __syncthreads();
    if (cnt > 0) {
#pragma unroll
        for (int q = 0; q < NF; ++q) {
            T* fb = sm + static_cast<size_t>(lib) * NF * pitch + q * pitch;   // cnt > 0 implies lib < lpb
#pragma unroll
            for (int k = 0; k < K; ++k)
                if (k < cnt) {
                    const int p = start + k;
                    fb[p + (p >> 5)] = JR[q][k];
                }
        }
    }
    __syncthreads();
    RedAcc<T> red{T(0), T(0)};
    for (int l = 0; l < lpb; ++l) {
        const int gl = line0 + l;
        if (gl >= nlines) break;
        const T* src = sm + static_cast<size_t>(l) * NF * pitch;
        for (int base = 0; base < n; base += U * blockDim.x) {
            T aux[U][Op::NA];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int p = base + u * blockDim.x + tid;
                if (p < n) op.fetch(gl, p, aux[u]);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int p = base + u * blockDim.x + tid;
                if (p < n) {
                    T h[NF];
#pragma unroll
                    for (int q = 0; q < NF; ++q) h[q] = src[q * pitch + p + (p >> 5)];
                    op.put(gl, p, h, aux[u], red);
                }
            }
        }
    }
    if (Op::kReduce) block_reduce_store<T>(red, red_slots);
}

template <typename T, int M, int K, class Op>
__global__ void __launch_bounds__(1024)
rows_kernel(const __grid_constant__ LineParams<T> lp, const Op op, int nlines, int tl_log2, int lpb,
            int pitch, unsigned long long* red_slots) {
    extern __shared__ __align__(16) unsigned char sm_rows[];
    rows_body<T, M, K, Op>(lp, op, nlines, tl_log2, lpb, pitch, static_cast<int>(blockIdx.x) * lpb,
                           reinterpret_cast<T*>(sm_rows), red_slots);
}

// =========================================================================================
// Rows, FP32, persistent and pipelined.  A block owns one line per iteration with K = KT
// positions per thread (TL = n / K threads; the launch uses K = 16) and loops over lines
// blockIdx.x, +gridDim.x, ...
// The staged input fields of the next line arrive by cp.async (16-byte chunks, swizzled) into
// the other half of a double buffer while the current line is swept; the epilogue's auxiliary
// fields of the current line are fetched the same way during the sweep.  Window reads and the
// epilogue work on 128-bit chunks; outputs are stored from registers.
// Requires n % 512 == 0, 1024 <= n <= 8192, 16-byte aligned rows, and the staged lines in
// shared memory.
// =========================================================================================
__device__ __forceinline__ float comp4(const float4& v, int e) {
    return e == 0 ? v.x : (e == 1 ? v.y : (e == 2 ? v.z : v.w));
}
__device__ __forceinline__ void set4(float4& v, int e, float x) {
    if (e == 0) v.x = x;
    else if (e == 1) v.y = x;
    else if (e == 2) v.z = x;
    else v.w = x;
}

template <int M, class Op, int KT = 16>
__global__ void __launch_bounds__(512, 1)
rows_pipe_kernel(const __grid_constant__ LineParams<float> lp, const __grid_constant__ PackedStencil pw, const Op op,
                 int nlines, long long ld, unsigned long long* red_slots, int rev) {
    using T = float;
    constexpr int K = KT, V = 4, KC = K / V, H = M / 2, WC = KC + 2;
    static_assert(K % V == 0 && K >= 8, "whole 16-byte chunks per thread, at least one wall stencil");
    constexpr int NS = Op::NS, NA = Op::NA, NF = Op::NF, NO = Op::NO;
    // two swept fields (pass 2): their stencil and recurrence steps run as fma.rn.f32x2 pairs
    constexpr bool kPack = NF == 2;
    using PL = Lanes<2>;
    extern __shared__ __align__(128) unsigned char sm_rows_pipe[];
    float4* sm = reinterpret_cast<float4*>(sm_rows_pipe);
    __shared__ T s_scan[16][2 + 2 * NF];   // per-warp segments: D_f, D_b, A_f[NF], A_b[NF]
    __shared__ T s_bnd[2 * NF];            // carries / B values of the line (FP64 solve)

    const int n = lp.n;
    const int nch = n / V;
    const int TL = blockDim.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, wpl = TL >> 5;
    const bool periodic = lp.bc == BC_PERIODIC;
    const T d = lp.d;
    const int start = tid * K;
    T D = T(1);
#pragma unroll
    for (int k = 0; k < K; ++k) D *= d;
    const T pl = dev_exp(-lp.nu * T(periodic ? start : start - 1));
    const T pr = dev_exp(-lp.nu * T(periodic ? n - start - K : n - start - K - 1));

    auto stage_buf = [&](int sb, int f) { return sm + (static_cast<size_t>(sb) * NS + f) * nch; };
    auto aux_buf = [&](int f) { return sm + (static_cast<size_t>(2 * NS) + f) * nch; };
    auto issue_staged = [&](int ln, int sb) {
#pragma unroll
        for (int f = 0; f < NS; ++f) {
            const float4* src = reinterpret_cast<const float4*>(op.s[f] + ln * ld);
            float4* dst = stage_buf(sb, f);
            for (int c = tid; c < nch; c += TL) cp_async16(dst + swz(c), src + c);
        }
    };

    // rev = 1 takes the lines from the last one up (the block order of the pass that ran before
    // decides which end of the field is still in L2)
    auto phys = [&](int l) { return rev ? nlines - 1 - l : l; };
    RedAcc<T> red{T(0), T(0)};
    int li = blockIdx.x;
    if (li < nlines) issue_staged(phys(li), 0);
    cp_async_commit();
    for (int it = 0; li < nlines; ++it, li += gridDim.x) {
        const int line = phys(li);
        const int sb = it & 1;
        cp_async_wait<0>();          // this line's staged fields (the only group in flight)
        __syncthreads();             // ... visible to all; every warp is done with the last line
        // auxiliary fields of this line, then the staged fields of the next line
#pragma unroll
        for (int f = 0; f < NA; ++f) {
            const float4* src = reinterpret_cast<const float4*>(op.a[f] + line * ld);
            float4* dst = aux_buf(f);
            for (int c = tid; c < nch; c += TL) cp_async16(dst + swz(c), src + c);
        }
        cp_async_commit();
        const int next = li + gridDim.x;
        if (next < nlines) issue_staged(phys(next), sb ^ 1);
        cp_async_commit();

        // ---- window (prologue applied) from chunks start/V - 1 .. start/V + KC ----
        T fw[NF][WC * V];
#pragma unroll
        for (int j = 0; j < WC; ++j) {
            int c = start / V - 1 + j;
            if (periodic) c = c < 0 ? c + nch : (c >= nch ? c - nch : c);
            else c = c < 0 ? 0 : (c >= nch ? nch - 1 : c);
            float4 raw[NS];
#pragma unroll
            for (int f = 0; f < NS; ++f) raw[f] = stage_buf(sb, f)[swz(c)];
#pragma unroll
            for (int e = 0; e < V; ++e) {
                T sv[NS], fv[NF];
#pragma unroll
                for (int f = 0; f < NS; ++f) sv[f] = comp4(raw[f], e);
                op.prologue(sv, fv);
#pragma unroll
                for (int q = 0; q < NF; ++q) fw[q][j * V + e] = fv[q];
            }
        }
        T JL[kPack ? 1 : NF][K], JR[kPack ? 1 : NF][K], aL[NF], aR[NF];
        unsigned long long JL2[kPack ? K : 1], JR2[kPack ? K : 1];   // packed J (then outputs)
        // J^L_j, J^R_j of the wall positions of a non-periodic line (shifted wall stencils, Sec. 3.2
        // reading), from the thread's own window: nodes 0..M of the first chunk sit at window
        // indices H + o, nodes N-M..N of the last chunk at K - 1 - M + H + o.  Same operations in
        // the same order as local_integrals.
        auto wall_integrals = [&](const T* win, T (&jlo)[K], T (&jro)[K]) {
            if (start == 0) {
#pragma unroll
                for (int k = 0; k < H; ++k) {   // j = k < H
                    T jl = T(0), jr = T(0);
#pragma unroll
                    for (int o = 0; o <= M; ++o) {
                        const T v = win[H + o];
                        if (k >= 1) jl = fma(lp.wlA[k - 1][o], v, jl);
                        jr = fma(lp.wrA[k][o], v, jr);
                    }
                    jlo[k] = jl;
                    jro[k] = jr;
                }
            }
            if (start + K == n) {
#pragma unroll
                for (int k = K - H; k < K; ++k) {   // j = start + k >= jb = n - H
                    T jl = T(0), jr = T(0);
#pragma unroll
                    for (int o = 0; o <= M; ++o) {
                        const T v = win[K - 1 - M + H + o];
                        jl = fma(lp.wlB[k - (K - H)][o], v, jl);
                        if (k < K - 1) jr = fma(lp.wrB[k - (K - H)][o], v, jr);
                    }
                    jlo[k] = jl;
                    jro[k] = jr;
                }
            }
        };
        if constexpr (kPack) {
            unsigned long long win2[K + M];
#pragma unroll
            for (int i = 0; i < K + M; ++i) win2[i] = PL::pack(fw[0][V - H + i], fw[1][V - H + i]);
#pragma unroll
            for (int k = 0; k < K; ++k) {
                unsigned long long jl = PL::fma(pw.wl[0], win2[k], PL::zero());
                unsigned long long jr = PL::fma(pw.wr[0], win2[k], PL::zero());
#pragma unroll
                for (int o = 1; o <= M; ++o) {
                    jl = PL::fma(pw.wl[o], win2[k + o], jl);
                    jr = PL::fma(pw.wr[o], win2[k + o], jr);
                }
                JL2[k] = jl;
                JR2[k] = jr;
            }
            if (!periodic) {
                // chunks touching a wall: the shifted wall stencils, field by field (as
                // local_integrals), from the thread's own packed window: nodes 0..M of the first
                // chunk sit at window indices H + o, nodes N-M..N of the last chunk at
                // K - 1 - M + H + o (the prologue is not evaluated again)
                if (start == 0) {
#pragma unroll
                    for (int k = 0; k < H; ++k) {   // j = k < H
                        T jl[2] = {T(0), T(0)}, jr[2] = {T(0), T(0)};
#pragma unroll
                        for (int q = 0; q < 2; ++q) {
#pragma unroll
                            for (int o = 0; o <= M; ++o) {
                                const T v = PL::get(win2[H + o], q);
                                if (k >= 1) jl[q] = fma(lp.wlA[k - 1][o], v, jl[q]);
                                jr[q] = fma(lp.wrA[k][o], v, jr[q]);
                            }
                        }
                        JL2[k] = PL::pack(jl[0], jl[1]);
                        JR2[k] = PL::pack(jr[0], jr[1]);
                    }
                }
                if (start + K == n) {
#pragma unroll
                    for (int k = K - H; k < K; ++k) {   // j = start + k >= jb = n - H
                        T jl[2] = {T(0), T(0)}, jr[2] = {T(0), T(0)};
#pragma unroll
                        for (int q = 0; q < 2; ++q) {
#pragma unroll
                            for (int o = 0; o <= M; ++o) {
                                const T v = PL::get(win2[K - 1 - M + H + o], q);
                                jl[q] = fma(lp.wlB[k - (K - H)][o], v, jl[q]);
                                if (k < K - 1) jr[q] = fma(lp.wrB[k - (K - H)][o], v, jr[q]);
                            }
                        }
                        JL2[k] = PL::pack(jl[0], jl[1]);
                        JR2[k] = PL::pack(jr[0], jr[1]);
                    }
                }
            }
            const unsigned long long d2 = PL::splat(d);
            unsigned long long a = PL::zero(), b = PL::zero();
#pragma unroll
            for (int k = 0; k < K; ++k) a = PL::fma(d2, a, JL2[k]);
#pragma unroll
            for (int k = K - 1; k >= 0; --k) b = PL::fma(d2, b, JR2[k]);
#pragma unroll
            for (int q = 0; q < NF; ++q) {
                aL[q] = PL::get(a, q);
                aR[q] = PL::get(b, q);
            }
        } else {
#pragma unroll
            for (int q = 0; q < NF; ++q) {
                T win[K + M];
#pragma unroll
                for (int i = 0; i < K + M; ++i) win[i] = fw[q][V - H + i];
#pragma unroll
                for (int k = 0; k < K; ++k) {   // interior stencil (as local_integrals)
                    T jl = T(0), jr = T(0);
#pragma unroll
                    for (int o = 0; o <= M; ++o) {
                        jl = fma(lp.wl[o], win[k + o], jl);
                        jr = fma(lp.wr[o], win[k + o], jr);
                    }
                    JL[q][k] = jl;
                    JR[q][k] = jr;
                }
                if (!periodic) wall_integrals(win, JL[q], JR[q]);
                chunk_aggregates<T, K>(d, K, JL[q], JR[q], aL[q], aR[q]);
            }
        }

        // ---- scan of the chunk segments: shuffles inside each warp ----
        T Df = D, Db = D, Af[NF], Ab[NF];
#pragma unroll
        for (int q = 0; q < NF; ++q) {
            Af[q] = aL[q];
            Ab[q] = aR[q];
        }
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const T dpf = __shfl_up_sync(kFull, Df, o);
            const T dpb = __shfl_down_sync(kFull, Db, o);
#pragma unroll
            for (int q = 0; q < NF; ++q) {
                const T apf = __shfl_up_sync(kFull, Af[q], o);
                const T apb = __shfl_down_sync(kFull, Ab[q], o);
                if (lane >= o) Af[q] = fma(apf, Df, Af[q]);
                if (lane + o < 32) Ab[q] = fma(apb, Db, Ab[q]);
            }
            if (lane >= o) Df = dpf * Df;
            if (lane + o < 32) Db = dpb * Db;
        }
        T Dxf = __shfl_up_sync(kFull, Df, 1), Dxb = __shfl_down_sync(kFull, Db, 1);
        T Axf[NF], Axb[NF];
#pragma unroll
        for (int q = 0; q < NF; ++q) {
            Axf[q] = __shfl_up_sync(kFull, Af[q], 1);
            Axb[q] = __shfl_down_sync(kFull, Ab[q], 1);
            if (lane == 0) Axf[q] = T(0);
            if (lane == 31) Axb[q] = T(0);
        }
        if (lane == 0) Dxf = T(1);
        if (lane == 31) Dxb = T(1);
        if (lane == 31) {
            s_scan[warp][0] = Df;
#pragma unroll
            for (int q = 0; q < NF; ++q) s_scan[warp][2 + q] = Af[q];
        }
        if (lane == 0) {
            s_scan[warp][1] = Db;
#pragma unroll
            for (int q = 0; q < NF; ++q) s_scan[warp][2 + NF + q] = Ab[q];
        }
        __syncthreads();
        // ---- warp 0 scans the warp segments (log depth) and solves the boundary system ----
        if (warp == 0) {
            const bool has = lane < wpl;
            T fD = has ? s_scan[lane][0] : T(1);
            T bD = has ? s_scan[lane][1] : T(1);
            T fA[NF], bA[NF];
#pragma unroll
            for (int q = 0; q < NF; ++q) {
                fA[q] = has ? s_scan[lane][2 + q] : T(0);
                bA[q] = has ? s_scan[lane][2 + NF + q] : T(0);
            }
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const T pfD = __shfl_up_sync(kFull, fD, o);
                const T pbD = __shfl_down_sync(kFull, bD, o);
#pragma unroll
                for (int q = 0; q < NF; ++q) {
                    const T pf = __shfl_up_sync(kFull, fA[q], o);
                    const T pb = __shfl_down_sync(kFull, bA[q], o);
                    if (lane >= o) fA[q] = fma(pf, fD, fA[q]);
                    if (lane + o < 32) bA[q] = fma(pb, bD, bA[q]);
                }
                if (lane >= o) fD = pfD * fD;
                if (lane + o < 32) bD = pbD * bD;
            }
            T exF[NF], exB[NF], totF[NF], totB[NF];
#pragma unroll
            for (int q = 0; q < NF; ++q) {
                exF[q] = __shfl_up_sync(kFull, fA[q], 1);
                exB[q] = __shfl_down_sync(kFull, bA[q], 1);
                totF[q] = __shfl_sync(kFull, fA[q], 31);
                totB[q] = __shfl_sync(kFull, bA[q], 0);
                if (lane == 0) exF[q] = T(0);
                if (lane + 1 >= wpl) exB[q] = T(0);
            }
            __syncwarp();
            if (has) {
#pragma unroll
                for (int q = 0; q < NF; ++q) {
                    s_scan[lane][2 + q] = exF[q];
                    s_scan[lane][2 + NF + q] = exB[q];
                }
            }
            // one FP64 2x2 boundary solve per line and field (Eq. homogeneous and analogues);
            // lane q solves field q
#pragma unroll
            for (int q = 0; q < NF; ++q) {
                if (lane == q) {
                    const double I0 = static_cast<double>(totB[q]);
                    const double IN = static_cast<double>(totF[q]);
                    double a, b;
                    if (periodic) {
                        a = IN * lp.inv1mmu;
                        b = I0 * lp.inv1mmu;
                    } else {
                        a = lp.bAA * I0 + lp.bAB * IN;
                        b = lp.bBA * I0 + lp.bBB * IN;
                    }
                    s_bnd[q] = static_cast<T>(a);
                    s_bnd[NF + q] = static_cast<T>(b);
                }
            }
        }
        __syncthreads();
        T pF[NF], pB[NF], xl[NF], xr[NF];
#pragma unroll
        for (int q = 0; q < NF; ++q) {
            pF[q] = s_scan[warp][2 + q];
            pB[q] = s_scan[warp][2 + NF + q];
            xl[q] = s_bnd[q];
            xr[q] = s_bnd[NF + q];
        }
        const bool wallL = !periodic && start == 0, wallR = !periodic && start + K == n;
        T cl[NF], cr[NF];
#pragma unroll
        for (int q = 0; q < NF; ++q) {
            const T ax = fma(pF[q], Dxf, Axf[q]);
            const T bx = fma(pB[q], Dxb, Axb[q]);
            cl[q] = wallL ? T(0) : fma(pl, xl[q], ax);   // at a wall, P^L_0 = B_a is injected instead
            cr[q] = wallR ? T(0) : fma(pr, xr[q], bx);   // ... and P^R_N = B_b
        }
        if constexpr (kPack) {
            if (wallL) JL2[0] = PL::add(JL2[0], PL::pack(xl[0], xl[1]));
            if (wallR) JR2[K - 1] = PL::add(JR2[K - 1], PL::pack(xr[0], xr[1]));
            const unsigned long long d2 = PL::splat(d);
            unsigned long long p = PL::pack(cr[0], cr[1]);
#pragma unroll
            for (int k = K - 1; k >= 0; --k) {
                p = PL::fma(d2, p, JR2[k]);
                JR2[k] = p;
            }
            unsigned long long qq = PL::pack(cl[0], cl[1]);
#pragma unroll
            for (int k = 0; k < K; ++k) {
                qq = PL::fma(d2, qq, JL2[k]);
                JR2[k] = PL::add(JR2[k], qq);
            }
        } else {
#pragma unroll
            for (int q = 0; q < NF; ++q) {
                if (wallL) JL[q][0] += xl[q];
                if (wallR) JR[q][K - 1] += xr[q];
                chunk_finish<T, K>(d, K, cl[q], cr[q], JL[q], JR[q]);
            }
        }

        // ---- epilogue on this thread's own chunks ----
        if constexpr (NA > 0) {
            cp_async_wait<1>();      // this line's auxiliary group is complete
            __syncthreads();
        }
#pragma unroll
        for (int kc = 0; kc < KC; ++kc) {
            const int c = start / V + kc;
            float4 sraw[NS], araw[NA > 0 ? NA : 1], outv[NO];
#pragma unroll
            for (int f = 0; f < NS; ++f) sraw[f] = stage_buf(sb, f)[swz(c)];
#pragma unroll
            for (int f = 0; f < NA; ++f) araw[f] = aux_buf(f)[swz(c)];
#pragma unroll
            for (int e = 0; e < V; ++e) {
                T h[NF], sv[NS], av[NA > 0 ? NA : 1], ov[NO];
#pragma unroll
                for (int q = 0; q < NF; ++q) {
                    if constexpr (kPack) h[q] = PL::get(JR2[kc * V + e], q);
                    else h[q] = JR[q][kc * V + e];
                }
#pragma unroll
                for (int f = 0; f < NS; ++f) sv[f] = comp4(sraw[f], e);
#pragma unroll
                for (int f = 0; f < NA; ++f) av[f] = comp4(araw[f], e);
                if constexpr (NA == 0) av[0] = T(0);
                op.epilogue(h, sv, av, ov, red);
#pragma unroll
                for (int o = 0; o < NO; ++o) set4(outv[o], e, ov[o]);
            }
#pragma unroll
            for (int o = 0; o < NO; ++o) reinterpret_cast<float4*>(op.o[o] + line * ld)[c] = outv[o];
        }
    }
    cp_async_wait<0>();
    if (Op::kReduce) block_reduce_store<T>(red, red_slots);
}

// =========================================================================================
// Rows, FP32, persistent and pipelined, one line split over a cluster of C blocks (the kernel above
// when C = 1; C = 2 here; the cluster's blocks are consecutive in x): block rank r owns the slice
// [r n/C, (r+1) n/C) with K = 16 positions per thread (TL = n / (16 C) threads).  Clusters loop
// over lines cluster_id, + number of clusters, ...  The staged input fields of the next line's
// slice, with one 16-byte chunk of halo on each side, arrive by cp.async (16-byte chunks,
// swizzled within 128-byte lines) into the other half of a double buffer while the current line
// is swept; the epilogue's auxiliary fields of the current slice are fetched the same way.
// Window reads and the epilogue work on 128-bit chunks; outputs are stored from registers.
// With C > 1 the blocks of a cluster exchange their slice segments (decay, left and right
// aggregates) through distributed shared memory once per line, so every block composes the
// carry entering its slice and the line totals of the boundary solve from the same values in the
// same order.  C = 2 serves lines whose staged fields do not fit one block (16384 nodes, or four
// staged fields of 8192 nodes).
// Requires n % (512 C) == 0, 1024 <= n <= 8192 C, TL <= 512, 16-byte aligned rows.
// =========================================================================================
// Thread-block cluster primitives (sm_90 and later).
__device__ __forceinline__ unsigned cluster_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void cluster_barrier() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// Load a float from the shared memory of block `rank` of this cluster at the address of `local`.
__device__ __forceinline__ float ld_cluster_f32(const float* local, unsigned rank) {
    unsigned remote;
    float v;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(static_cast<unsigned>(__cvta_generic_to_shared(local))), "r"(rank));
    asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(remote) : "memory");
    return v;
}

// Index of local chunk lc (-1 .. nchl) in a staged slice: the nchl swizzled chunks of the slice
// from the buffer's start (so every group of 8 chunks is one aligned 128-byte line of the swizzle),
// then the left and the right halo chunk.
__device__ __forceinline__ int staged_index(int lc, int nchl) {
    return lc < 0 ? nchl : (lc >= nchl ? nchl + 1 : swz(lc));
}

template <int M, class Op, int C>
__global__ void __launch_bounds__(512, 1)
rows_cluster_kernel(const __grid_constant__ LineParams<float> lp, const __grid_constant__ PackedStencil pw, const Op op,
                    int nlines, long long ld, unsigned long long* red_slots) {
    using T = float;
    constexpr int K = 16, V = 4, KC = K / V, H = M / 2, WC = KC + 2;
    constexpr int NS = Op::NS, NA = Op::NA, NF = Op::NF, NO = Op::NO;
    // two swept fields (pass 2): their stencil and recurrence steps run as fma.rn.f32x2 pairs
    constexpr bool kPack = NF == 2;
    using PL = Lanes<2>;
    extern __shared__ __align__(128) unsigned char sm_rows_pipe[];
    float4* sm = reinterpret_cast<float4*>(sm_rows_pipe);
    __shared__ T s_scan[16][2 + 2 * NF];   // per-warp segments: D_f, D_b, A_f[NF], A_b[NF]
    __shared__ T s_bnd[2 * NF];            // carries / B values of the line (FP64 solve)
    __shared__ T s_xch[2][1 + 2 * NF];     // this block's slice segment, by line parity (C > 1)

    const int n = lp.n;
    const int nch = n / V;                 // chunks of the line
    const int nchl = nch / C;              // chunks of this block's slice
    const int rank = C > 1 ? static_cast<int>(cluster_rank()) : 0;
    const int c0 = rank * nchl;            // first chunk of the slice
    const int slice0 = c0 * V;             // first position of the slice
    const int TL = blockDim.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, wpl = TL >> 5;
    const bool periodic = lp.bc == BC_PERIODIC;
    const T d = lp.d;
    const int lstart = tid * K;            // first position of the thread's chunk within the slice
    const int start = slice0 + lstart;     // ... within the line
    T D = T(1);
#pragma unroll
    for (int k = 0; k < K; ++k) D *= d;
    const T pl = dev_exp(-lp.nu * T(periodic ? start : start - 1));
    const T pr = dev_exp(-lp.nu * T(periodic ? n - start - K : n - start - K - 1));

    const int sbuf = nchl + 8;             // staged chunks per field: slice, two halo chunks, padding to
                                           // a multiple of 8 chunks (128-byte aligned buffers)
    auto stage_buf = [&](int sb, int f) { return sm + (static_cast<size_t>(sb) * NS + f) * sbuf; };
    auto aux_buf = [&](int f) { return sm + static_cast<size_t>(2 * NS) * sbuf + static_cast<size_t>(f) * nchl; };
    auto issue_staged = [&](int ln, int sb) {
#pragma unroll
        for (int f = 0; f < NS; ++f) {
            const float4* src = reinterpret_cast<const float4*>(op.s[f] + ln * ld);
            float4* dst = stage_buf(sb, f);
            for (int c = tid; c < nchl + 2; c += TL) {
                const int lc = c - 1;
                int gc = c0 + lc;
                if (periodic) gc = gc < 0 ? gc + nch : (gc >= nch ? gc - nch : gc);
                else gc = gc < 0 ? 0 : (gc >= nch ? nch - 1 : gc);
                cp_async16(dst + staged_index(lc, nchl), src + gc);
            }
        }
    };

    const int cid = C > 1 ? static_cast<int>(blockIdx.x) / C : static_cast<int>(blockIdx.x);
    const int ncl = C > 1 ? static_cast<int>(gridDim.x) / C : static_cast<int>(gridDim.x);
    RedAcc<T> red{T(0), T(0)};
    int line = cid;
    if (line < nlines) issue_staged(line, 0);
    cp_async_commit();
    for (int it = 0; line < nlines; ++it, line += ncl) {
        const int sb = it & 1;
        cp_async_wait<0>();          // this line's staged fields (the only group in flight)
        __syncthreads();             // ... visible to all; every warp is done with the last line
        // auxiliary fields of this slice, then the staged fields of the next line
#pragma unroll
        for (int f = 0; f < NA; ++f) {
            const float4* src = reinterpret_cast<const float4*>(op.a[f] + line * ld) + c0;
            float4* dst = aux_buf(f);
            for (int c = tid; c < nchl; c += TL) cp_async16(dst + swz(c), src + c);
        }
        cp_async_commit();
        const int next = line + ncl;
        if (next < nlines) issue_staged(next, sb ^ 1);
        cp_async_commit();

        // ---- window (prologue applied) from local chunks lstart/V - 1 .. lstart/V + KC ----
        T fw[NF][WC * V];
#pragma unroll
        for (int j = 0; j < WC; ++j) {
            const int idx = staged_index(lstart / V - 1 + j, nchl);
            float4 raw[NS];
#pragma unroll
            for (int f = 0; f < NS; ++f) raw[f] = stage_buf(sb, f)[idx];
#pragma unroll
            for (int e = 0; e < V; ++e) {
                T sv[NS], fv[NF];
#pragma unroll
                for (int f = 0; f < NS; ++f) sv[f] = comp4(raw[f], e);
                op.prologue(sv, fv);
#pragma unroll
                for (int q = 0; q < NF; ++q) fw[q][j * V + e] = fv[q];
            }
        }
        T JL[kPack ? 1 : NF][K], JR[kPack ? 1 : NF][K], aL[NF], aR[NF];
        unsigned long long JL2[kPack ? K : 1], JR2[kPack ? K : 1];   // packed J (then outputs)
        // J^L_j, J^R_j of the wall positions of a non-periodic line (shifted wall stencils, Sec. 3.2
        // reading), from the thread's own window: nodes 0..M of the first chunk sit at window
        // indices H + o, nodes N-M..N of the last chunk at K - 1 - M + H + o.  Same operations in
        // the same order as local_integrals.
        auto wall_integrals = [&](const T* win, T (&jlo)[K], T (&jro)[K]) {
            if (start == 0) {
#pragma unroll
                for (int k = 0; k < H; ++k) {   // j = k < H
                    T jl = T(0), jr = T(0);
#pragma unroll
                    for (int o = 0; o <= M; ++o) {
                        const T v = win[H + o];
                        if (k >= 1) jl = fma(lp.wlA[k - 1][o], v, jl);
                        jr = fma(lp.wrA[k][o], v, jr);
                    }
                    jlo[k] = jl;
                    jro[k] = jr;
                }
            }
            if (start + K == n) {
#pragma unroll
                for (int k = K - H; k < K; ++k) {   // j = start + k >= jb = n - H
                    T jl = T(0), jr = T(0);
#pragma unroll
                    for (int o = 0; o <= M; ++o) {
                        const T v = win[K - 1 - M + H + o];
                        jl = fma(lp.wlB[k - (K - H)][o], v, jl);
                        if (k < K - 1) jr = fma(lp.wrB[k - (K - H)][o], v, jr);
                    }
                    jlo[k] = jl;
                    jro[k] = jr;
                }
            }
        };
        if constexpr (kPack) {
            unsigned long long win2[K + M];
#pragma unroll
            for (int i = 0; i < K + M; ++i) win2[i] = PL::pack(fw[0][V - H + i], fw[1][V - H + i]);
#pragma unroll
            for (int k = 0; k < K; ++k) {
                unsigned long long jl = PL::fma(pw.wl[0], win2[k], PL::zero());
                unsigned long long jr = PL::fma(pw.wr[0], win2[k], PL::zero());
#pragma unroll
                for (int o = 1; o <= M; ++o) {
                    jl = PL::fma(pw.wl[o], win2[k + o], jl);
                    jr = PL::fma(pw.wr[o], win2[k + o], jr);
                }
                JL2[k] = jl;
                JR2[k] = jr;
            }
            if (!periodic) {
                // chunks touching a wall: the shifted wall stencils, field by field (as
                // local_integrals), from the thread's own packed window: nodes 0..M of the first
                // chunk sit at window indices H + o, nodes N-M..N of the last chunk at
                // K - 1 - M + H + o (the prologue is not evaluated again)
                if (start == 0) {
#pragma unroll
                    for (int k = 0; k < H; ++k) {   // j = k < H
                        T jl[2] = {T(0), T(0)}, jr[2] = {T(0), T(0)};
#pragma unroll
                        for (int q = 0; q < 2; ++q) {
#pragma unroll
                            for (int o = 0; o <= M; ++o) {
                                const T v = PL::get(win2[H + o], q);
                                if (k >= 1) jl[q] = fma(lp.wlA[k - 1][o], v, jl[q]);
                                jr[q] = fma(lp.wrA[k][o], v, jr[q]);
                            }
                        }
                        JL2[k] = PL::pack(jl[0], jl[1]);
                        JR2[k] = PL::pack(jr[0], jr[1]);
                    }
                }
                if (start + K == n) {
#pragma unroll
                    for (int k = K - H; k < K; ++k) {   // j = start + k >= jb = n - H
                        T jl[2] = {T(0), T(0)}, jr[2] = {T(0), T(0)};
#pragma unroll
                        for (int q = 0; q < 2; ++q) {
#pragma unroll
                            for (int o = 0; o <= M; ++o) {
                                const T v = PL::get(win2[K - 1 - M + H + o], q);
                                jl[q] = fma(lp.wlB[k - (K - H)][o], v, jl[q]);
                                if (k < K - 1) jr[q] = fma(lp.wrB[k - (K - H)][o], v, jr[q]);
                            }
                        }
                        JL2[k] = PL::pack(jl[0], jl[1]);
                        JR2[k] = PL::pack(jr[0], jr[1]);
                    }
                }
            }
            const unsigned long long d2 = PL::splat(d);
            unsigned long long a = PL::zero(), b = PL::zero();
#pragma unroll
            for (int k = 0; k < K; ++k) a = PL::fma(d2, a, JL2[k]);
#pragma unroll
            for (int k = K - 1; k >= 0; --k) b = PL::fma(d2, b, JR2[k]);
#pragma unroll
            for (int q = 0; q < NF; ++q) {
                aL[q] = PL::get(a, q);
                aR[q] = PL::get(b, q);
            }
        } else {
#pragma unroll
            for (int q = 0; q < NF; ++q) {
                T win[K + M];
#pragma unroll
                for (int i = 0; i < K + M; ++i) win[i] = fw[q][V - H + i];
#pragma unroll
                for (int k = 0; k < K; ++k) {   // interior stencil (as local_integrals)
                    T jl = T(0), jr = T(0);
#pragma unroll
                    for (int o = 0; o <= M; ++o) {
                        jl = fma(lp.wl[o], win[k + o], jl);
                        jr = fma(lp.wr[o], win[k + o], jr);
                    }
                    JL[q][k] = jl;
                    JR[q][k] = jr;
                }
                if (!periodic) wall_integrals(win, JL[q], JR[q]);
                chunk_aggregates<T, K>(d, K, JL[q], JR[q], aL[q], aR[q]);
            }
        }

        // ---- scan of the chunk segments: shuffles inside each warp ----
        T Df = D, Db = D, Af[NF], Ab[NF];
#pragma unroll
        for (int q = 0; q < NF; ++q) {
            Af[q] = aL[q];
            Ab[q] = aR[q];
        }
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const T dpf = __shfl_up_sync(kFull, Df, o);
            const T dpb = __shfl_down_sync(kFull, Db, o);
#pragma unroll
            for (int q = 0; q < NF; ++q) {
                const T apf = __shfl_up_sync(kFull, Af[q], o);
                const T apb = __shfl_down_sync(kFull, Ab[q], o);
                if (lane >= o) Af[q] = fma(apf, Df, Af[q]);
                if (lane + o < 32) Ab[q] = fma(apb, Db, Ab[q]);
            }
            if (lane >= o) Df = dpf * Df;
            if (lane + o < 32) Db = dpb * Db;
        }
        T Dxf = __shfl_up_sync(kFull, Df, 1), Dxb = __shfl_down_sync(kFull, Db, 1);
        T Axf[NF], Axb[NF];
#pragma unroll
        for (int q = 0; q < NF; ++q) {
            Axf[q] = __shfl_up_sync(kFull, Af[q], 1);
            Axb[q] = __shfl_down_sync(kFull, Ab[q], 1);
            if (lane == 0) Axf[q] = T(0);
            if (lane == 31) Axb[q] = T(0);
        }
        if (lane == 0) Dxf = T(1);
        if (lane == 31) Dxb = T(1);
        if (lane == 31) {
            s_scan[warp][0] = Df;
#pragma unroll
            for (int q = 0; q < NF; ++q) s_scan[warp][2 + q] = Af[q];
        }
        if (lane == 0) {
            s_scan[warp][1] = Db;
#pragma unroll
            for (int q = 0; q < NF; ++q) s_scan[warp][2 + NF + q] = Ab[q];
        }
        __syncthreads();
        // ---- warp 0 scans the warp segments (log depth) and solves the boundary system ----
        T exF[NF], exB[NF], totF[NF], totB[NF], exDf = T(1), exDb = T(1);
        if (warp == 0) {
            const bool has = lane < wpl;
            T fD = has ? s_scan[lane][0] : T(1);
            T bD = has ? s_scan[lane][1] : T(1);
            T fA[NF], bA[NF];
#pragma unroll
            for (int q = 0; q < NF; ++q) {
                fA[q] = has ? s_scan[lane][2 + q] : T(0);
                bA[q] = has ? s_scan[lane][2 + NF + q] : T(0);
            }
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const T pfD = __shfl_up_sync(kFull, fD, o);
                const T pbD = __shfl_down_sync(kFull, bD, o);
#pragma unroll
                for (int q = 0; q < NF; ++q) {
                    const T pf = __shfl_up_sync(kFull, fA[q], o);
                    const T pb = __shfl_down_sync(kFull, bA[q], o);
                    if (lane >= o) fA[q] = fma(pf, fD, fA[q]);
                    if (lane + o < 32) bA[q] = fma(pb, bD, bA[q]);
                }
                if (lane >= o) fD = pfD * fD;
                if (lane + o < 32) bD = pbD * bD;
            }
#pragma unroll
            for (int q = 0; q < NF; ++q) {
                exF[q] = __shfl_up_sync(kFull, fA[q], 1);
                exB[q] = __shfl_down_sync(kFull, bA[q], 1);
                totF[q] = __shfl_sync(kFull, fA[q], 31);
                totB[q] = __shfl_sync(kFull, bA[q], 0);
                if (lane == 0) exF[q] = T(0);
                if (lane + 1 >= wpl) exB[q] = T(0);
            }
            if constexpr (C > 1) {
                exDf = __shfl_up_sync(kFull, fD, 1);      // decay of the warps before this one
                exDb = __shfl_down_sync(kFull, bD, 1);    // ... and after it
                if (lane == 0) exDf = T(1);
                if (lane + 1 >= wpl) exDb = T(1);
                const T Dc = __shfl_sync(kFull, fD, 31);  // decay over the slice
                if (lane == 0) {
                    s_xch[it & 1][0] = Dc;
#pragma unroll
                    for (int q = 0; q < NF; ++q) {
                        s_xch[it & 1][1 + q] = totF[q];
                        s_xch[it & 1][1 + NF + q] = totB[q];
                    }
                }
            }
        }
        if constexpr (C > 1) {
            // the slice segments of the cluster's blocks, read by every block in rank order
            cluster_barrier();
            if (warp == 0) {
                T Ef[NF], Eb[NF], IN[NF], I0[NF];
#pragma unroll
                for (int q = 0; q < NF; ++q) Ef[q] = Eb[q] = IN[q] = I0[q] = T(0);
#pragma unroll
                for (int r = 0; r < C; ++r) {                     // forward: ranks in order
                    const T Dr = ld_cluster_f32(&s_xch[it & 1][0], r);
#pragma unroll
                    for (int q = 0; q < NF; ++q) {
                        const T Fr = ld_cluster_f32(&s_xch[it & 1][1 + q], r);
                        if (r < rank) Ef[q] = fma(Ef[q], Dr, Fr);
                        IN[q] = fma(IN[q], Dr, Fr);
                    }
                }
#pragma unroll
                for (int r = C - 1; r >= 0; --r) {                // backward: ranks in reverse
                    const T Dr = ld_cluster_f32(&s_xch[it & 1][0], r);
#pragma unroll
                    for (int q = 0; q < NF; ++q) {
                        const T Br = ld_cluster_f32(&s_xch[it & 1][1 + NF + q], r);
                        if (r > rank) Eb[q] = fma(Eb[q], Dr, Br);
                        I0[q] = fma(I0[q], Dr, Br);
                    }
                }
#pragma unroll
                for (int q = 0; q < NF; ++q) {
                    exF[q] = fma(Ef[q], exDf, exF[q]);   // carry entering the warp from the line start
                    exB[q] = fma(Eb[q], exDb, exB[q]);   // ... and from the line end
                    totF[q] = IN[q];
                    totB[q] = I0[q];
                }
            }
        }
        if (warp == 0) {
            __syncwarp();
            if (lane < wpl) {
#pragma unroll
                for (int q = 0; q < NF; ++q) {
                    s_scan[lane][2 + q] = exF[q];
                    s_scan[lane][2 + NF + q] = exB[q];
                }
            }
            // one FP64 2x2 boundary solve per line and field (Eq. homogeneous and analogues);
            // lane q solves field q
#pragma unroll
            for (int q = 0; q < NF; ++q) {
                if (lane == q) {
                    const double I0 = static_cast<double>(totB[q]);
                    const double IN = static_cast<double>(totF[q]);
                    double a, b;
                    if (periodic) {
                        a = IN * lp.inv1mmu;
                        b = I0 * lp.inv1mmu;
                    } else {
                        a = lp.bAA * I0 + lp.bAB * IN;
                        b = lp.bBA * I0 + lp.bBB * IN;
                    }
                    s_bnd[q] = static_cast<T>(a);
                    s_bnd[NF + q] = static_cast<T>(b);
                }
            }
        }
        __syncthreads();
        T pF[NF], pB[NF], xl[NF], xr[NF];
#pragma unroll
        for (int q = 0; q < NF; ++q) {
            pF[q] = s_scan[warp][2 + q];
            pB[q] = s_scan[warp][2 + NF + q];
            xl[q] = s_bnd[q];
            xr[q] = s_bnd[NF + q];
        }
        const bool wallL = !periodic && start == 0, wallR = !periodic && start + K == n;
        T cl[NF], cr[NF];
#pragma unroll
        for (int q = 0; q < NF; ++q) {
            const T ax = fma(pF[q], Dxf, Axf[q]);
            const T bx = fma(pB[q], Dxb, Axb[q]);
            cl[q] = wallL ? T(0) : fma(pl, xl[q], ax);   // at a wall, P^L_0 = B_a is injected instead
            cr[q] = wallR ? T(0) : fma(pr, xr[q], bx);   // ... and P^R_N = B_b
        }
        if constexpr (kPack) {
            if (wallL) JL2[0] = PL::add(JL2[0], PL::pack(xl[0], xl[1]));
            if (wallR) JR2[K - 1] = PL::add(JR2[K - 1], PL::pack(xr[0], xr[1]));
            const unsigned long long d2 = PL::splat(d);
            unsigned long long p = PL::pack(cr[0], cr[1]);
#pragma unroll
            for (int k = K - 1; k >= 0; --k) {
                p = PL::fma(d2, p, JR2[k]);
                JR2[k] = p;
            }
            unsigned long long qq = PL::pack(cl[0], cl[1]);
#pragma unroll
            for (int k = 0; k < K; ++k) {
                qq = PL::fma(d2, qq, JL2[k]);
                JR2[k] = PL::add(JR2[k], qq);
            }
        } else {
#pragma unroll
            for (int q = 0; q < NF; ++q) {
                if (wallL) JL[q][0] += xl[q];
                if (wallR) JR[q][K - 1] += xr[q];
                chunk_finish<T, K>(d, K, cl[q], cr[q], JL[q], JR[q]);
            }
        }

        // ---- epilogue on this thread's own chunks ----
        if constexpr (NA > 0) {
            cp_async_wait<1>();      // this line's auxiliary group is complete
            __syncthreads();
        }
#pragma unroll
        for (int kc = 0; kc < KC; ++kc) {
            const int c = lstart / V + kc;          // local chunk
            float4 sraw[NS], araw[NA > 0 ? NA : 1], outv[NO];
#pragma unroll
            for (int f = 0; f < NS; ++f) sraw[f] = stage_buf(sb, f)[swz(c)];
#pragma unroll
            for (int f = 0; f < NA; ++f) araw[f] = aux_buf(f)[swz(c)];
#pragma unroll
            for (int e = 0; e < V; ++e) {
                T h[NF], sv[NS], av[NA > 0 ? NA : 1], ov[NO];
#pragma unroll
                for (int q = 0; q < NF; ++q) {
                    if constexpr (kPack) h[q] = PL::get(JR2[kc * V + e], q);
                    else h[q] = JR[q][kc * V + e];
                }
#pragma unroll
                for (int f = 0; f < NS; ++f) sv[f] = comp4(sraw[f], e);
#pragma unroll
                for (int f = 0; f < NA; ++f) av[f] = comp4(araw[f], e);
                if constexpr (NA == 0) av[0] = T(0);
                op.epilogue(h, sv, av, ov, red);
#pragma unroll
                for (int o = 0; o < NO; ++o) set4(outv[o], e, ov[o]);
            }
#pragma unroll
            for (int o = 0; o < NO; ++o) reinterpret_cast<float4*>(op.o[o] + line * ld)[c0 + c] = outv[o];
        }
    }
    cp_async_wait<0>();
    // no block of a cluster leaves while another may still read its exchange slots
    if constexpr (C > 1) cluster_barrier();
    if (Op::kReduce) block_reduce_store<T>(red, red_slots);
}

// =========================================================================================
// Columns, FP32, persistent and pipelined.  A work item is one tile of R = 128 rows of a strip
// of 32 columns (each staged row is one 128-byte segment per field); items are visited
// strip-fastest so that concurrent blocks read adjacent segments of the same rows.  The rows
// [r0 - 3, r0 + R + 3) of the next item's staged fields arrive by cp.async while the current
// item is processed.  kFinal = false: tile aggregates (phase A); kFinal = true: the tile's
// results from the carries of the scan kernel (phase C).
// Phase A uses that a tile aggregate of J = (stencil applied to f) is the stencil weights
// applied to M+1 shifted recurrences of f: with window w[i] = f at start - M/2 + i,
//   sum_k d^{K-1-k} J^L_k = sum_o wl_o S_o,  S_0 = sum_k d^{K-1-k} w[k],
//                                            S_{o+1} = d S_o - d^K w[o] + w[K+o];
//   sum_k d^k J^R_k      = sum_o wr_o R_o,  R_M = sum_k d^k w[k+M],
//                                            R_o = w[o] + d (R_{o+1} - d^{K-1} w[K+o]).
// Requires nlines % 32 == 0, n >= 256, 16-byte aligned rows.
// =========================================================================================
template <int M, class Op, bool kFinal>
__global__ void __launch_bounds__(256, 2)
cols_pipe_kernel(const __grid_constant__ LineParams<float> lp, const Op op, int nlines, long long ld, int tiles,
                 float* __restrict__ aggL, float* __restrict__ aggR, const float* __restrict__ carL,
                 const float* __restrict__ carR, unsigned long long* red_slots) {
    using T = float;
    constexpr int KY = 16, WY = 8, R = KY * WY, HR = kMaxM / 2, ROWS = R + 2 * HR, H = M / 2;
    constexpr int NS = Op::NS, NF = Op::NF, NO = Op::NO;
    extern __shared__ __align__(128) unsigned char sm_cols_pipe[];
    float* sm = reinterpret_cast<float*>(sm_cols_pipe);   // [2][NS][ROWS][32]
    __shared__ T sD[WY][32];
    __shared__ T sL[NF][WY][32];
    __shared__ T sR[NF][WY][32];
    const int lane = threadIdx.x & 31, wy = threadIdx.x >> 5;
    const int n = lp.n, N = lp.N, jb = lp.N - H + 1;
    const bool periodic = lp.bc == BC_PERIODIC;
    const T d = lp.d;
    const int nstrips = nlines >> 5;
    const int items = nstrips * tiles;
    T DK = T(1);
#pragma unroll
    for (int k = 0; k < KY - 1; ++k) DK *= d;
    const T DK1 = DK;          // d^{KY-1}
    DK *= d;                   // d^{KY}

    auto buf = [&](int sb, int f) { return sm + (static_cast<size_t>(sb) * NS + f) * ROWS * 32; };
    auto issue = [&](int itm, int sb) {
        const int strip = itm % nstrips, tile = itm / nstrips;
        const int r0 = tile * R - HR;
#pragma unroll
        for (int f = 0; f < NS; ++f) {
            const T* base = op.s[f] + strip * 32;
            float* dst = buf(sb, f);
            for (int idx = threadIdx.x; idx < ROWS * 8; idx += blockDim.x) {
                const int rr = idx >> 3, ch = idx & 7;
                const int row = fold_pos(r0 + rr, n, periodic);
                cp_async16(dst + rr * 32 + ch * 4, base + row * ld + ch * 4);
            }
        }
    };

    RedAcc<T> red{T(0), T(0)};
    int item = blockIdx.x;
    if (item < items) issue(item, 0);
    cp_async_commit();
    for (int it = 0; item < items; ++it, item += gridDim.x) {
        const int sb = it & 1;
        cp_async_wait<0>();
        __syncthreads();
        const int nxt = item + gridDim.x;
        if (nxt < items) issue(nxt, sb ^ 1);
        cp_async_commit();

        const int strip = item % nstrips, tile = item / nstrips;
        const int line = strip * 32 + lane;
        const int r0 = tile * R - HR;
        const int start = tile * R + wy * KY;
        int cnt = n - start;
        cnt = cnt < 0 ? 0 : (cnt > KY ? KY : cnt);
        // window of swept values: win[q][i] at position start - H + i
        T win[NF][KY + M];
#pragma unroll
        for (int i = 0; i < KY + M; ++i) {
            const int rr = wy * KY + HR - H + i;
            T sv[NS], fv[NF];
#pragma unroll
            for (int f = 0; f < NS; ++f) sv[f] = buf(sb, f)[rr * 32 + lane];
            op.prologue(sv, fv);
#pragma unroll
            for (int q = 0; q < NF; ++q) win[q][i] = fv[q];
        }
        T D = T(1);
#pragma unroll
        for (int k = 0; k < KY; ++k)
            if (k < cnt) D *= d;
        const bool interior = (cnt == KY) && (periodic || (start >= H && start + KY - 1 <= N - H));
        // wall values injected at the end nodes in phase C (from the scan kernel), 0 otherwise
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
        auto at = [&](int p, int q) {
            const int rr = p - r0;
            T sv[NS], fv[NF];
            if (rr >= 0 && rr < ROWS) {
#pragma unroll
                for (int f = 0; f < NS; ++f) sv[f] = buf(sb, f)[rr * 32 + lane];
            } else {
#pragma unroll
                for (int f = 0; f < NS; ++f) sv[f] = op.s[f][static_cast<long long>(p) * ld + line];
            }
            op.prologue(sv, fv);
            return fv[q];
        };
        // J^L / J^R at chunk position k (j = start + k), wall stencils and injections included
        auto jl = [&](int q, int k) {
            const int j = start + k;
            T a = T(0);
            if (!periodic && j < H) {
                if (j == 0) return injL[q];
                for (int o = 0; o <= M; ++o) a = fma(lp.wlA[j - 1][o], at(o, q), a);
            } else if (!periodic && j >= jb) {
                for (int o = 0; o <= M; ++o) a = fma(lp.wlB[j - jb][o], at(N - M + o, q), a);
            } else {
#pragma unroll
                for (int o = 0; o <= M; ++o) a = fma(lp.wl[o], win[q][k + o], a);
            }
            return a;
        };
        auto jr = [&](int q, int k) {
            const int j = start + k;
            T a = T(0);
            if (!periodic && j < H) {
                for (int o = 0; o <= M; ++o) a = fma(lp.wrA[j][o], at(o, q), a);
            } else if (!periodic && j >= jb) {
                if (j == N) return injR[q];
                for (int o = 0; o <= M; ++o) a = fma(lp.wrB[j - jb][o], at(N - M + o, q), a);
            } else {
#pragma unroll
                for (int o = 0; o <= M; ++o) a = fma(lp.wr[o], win[q][k + o], a);
            }
            return a;
        };

        // ---- chunk aggregates ----
        T aL[NF], aR[NF];
#pragma unroll
        for (int q = 0; q < NF; ++q) {
            if (interior) {
                T S = T(0);
#pragma unroll
                for (int k = 0; k < KY; ++k) S = fma(d, S, win[q][k]);
                T a = lp.wl[0] * S;
#pragma unroll
                for (int o = 0; o < M; ++o) {
                    S = fma(d, S, fma(-DK, win[q][o], win[q][KY + o]));
                    a = fma(lp.wl[o + 1], S, a);
                }
                T Rr = T(0);
#pragma unroll
                for (int k = KY - 1; k >= 0; --k) Rr = fma(d, Rr, win[q][k + M]);
                T b = lp.wr[M] * Rr;
#pragma unroll
                for (int o = M - 1; o >= 0; --o) {
                    Rr = fma(d, fma(-DK1, win[q][KY + o], Rr), win[q][o]);
                    b = fma(lp.wr[o], Rr, b);
                }
                aL[q] = a;
                aR[q] = b;
            } else {
                T a = T(0), b = T(0);
#pragma unroll
                for (int k = 0; k < KY; ++k)
                    if (k < cnt) a = fma(d, a, jl(q, k));
#pragma unroll
                for (int k = KY - 1; k >= 0; --k)
                    if (k < cnt) b = fma(d, b, jr(q, k));
                aL[q] = a;
                aR[q] = b;
            }
        }
        sD[wy][lane] = D;
#pragma unroll
        for (int q = 0; q < NF; ++q) {
            sL[q][wy][lane] = aL[q];
            sR[q][wy][lane] = aR[q];
        }
        __syncthreads();
        if constexpr (!kFinal) {
            if (wy == 0) {
#pragma unroll
                for (int q = 0; q < NF; ++q) {
                    T a = T(0), b = T(0);
#pragma unroll
                    for (int i = 0; i < WY; ++i) a = fma(a, sD[i][lane], sL[q][i][lane]);
#pragma unroll
                    for (int i = WY - 1; i >= 0; --i) b = fma(b, sD[i][lane], sR[q][i][lane]);
                    const size_t o = (static_cast<size_t>(q) * tiles + tile) * nlines + line;
                    aggL[o] = a;
                    aggR[o] = b;
                }
            }
        } else {
            T out[NF][KY];
#pragma unroll
            for (int q = 0; q < NF; ++q) {
                const size_t o = (static_cast<size_t>(q) * tiles + tile) * nlines + line;
                T cl = (!periodic && tile == 0) ? T(0) : carL[o];
                T cr = (!periodic && tile == tiles - 1) ? T(0) : carR[o];
#pragma unroll
                for (int i = 0; i < WY; ++i)
                    if (i < wy) cl = fma(cl, sD[i][lane], sL[q][i][lane]);
#pragma unroll
                for (int i = WY - 1; i >= 0; --i)
                    if (i > wy) cr = fma(cr, sD[i][lane], sR[q][i][lane]);
                // second pass: P^R backward, then P^L forward added (Eq. IL / IR from the carries)
                T p = cr;
                if (interior) {
#pragma unroll
                    for (int k = KY - 1; k >= 0; --k) {
                        T a = T(0);
#pragma unroll
                        for (int o2 = 0; o2 <= M; ++o2) a = fma(lp.wr[o2], win[q][k + o2], a);
                        p = fma(d, p, a);
                        out[q][k] = p;
                    }
                    T s2 = cl;
#pragma unroll
                    for (int k = 0; k < KY; ++k) {
                        T a = T(0);
#pragma unroll
                        for (int o2 = 0; o2 <= M; ++o2) a = fma(lp.wl[o2], win[q][k + o2], a);
                        s2 = fma(d, s2, a);
                        out[q][k] += s2;
                    }
                } else {
#pragma unroll
                    for (int k = KY - 1; k >= 0; --k)
                        if (k < cnt) {
                            p = fma(d, p, jr(q, k));
                            out[q][k] = p;
                        }
                    T s2 = cl;
#pragma unroll
                    for (int k = 0; k < KY; ++k)
                        if (k < cnt) {
                            s2 = fma(d, s2, jl(q, k));
                            out[q][k] += s2;
                        }
                }
            }
            T* ob[NO];
#pragma unroll
            for (int o = 0; o < NO; ++o) ob[o] = op.o[o] + static_cast<long long>(start) * ld + line;
            const float* sbase = buf(sb, 0) + (wy * KY + HR) * 32 + lane;
#pragma unroll
            for (int k = 0; k < KY; ++k) {
                if (k < cnt) {
                    T h[NF], sv[NS], av[1] = {T(0)}, ov[NO];
#pragma unroll
                    for (int q = 0; q < NF; ++q) h[q] = out[q][k];
#pragma unroll
                    for (int f = 0; f < NS; ++f) sv[f] = sbase[static_cast<size_t>(f) * ROWS * 32 + k * 32];
                    op.epilogue(h, sv, av, ov, red);
#pragma unroll
                    for (int o = 0; o < NO; ++o) *ob[o] = ov[o];
                }
#pragma unroll
                for (int o = 0; o < NO; ++o) ob[o] += ld;
            }
        }
    }
    cp_async_wait<0>();
    if (Op::kReduce) block_reduce_store<T>(red, red_slots);
}

// =========================================================================================
// Columns.  Block = 32 lanes (32 adjacent columns, so every access is a 128 B row segment in
// FP32) x WY warps; a tile is R = WY * KY positions of those columns.  Phase A reduces each
// tile to its two segments, phase B scans the tile segments down each column (FP64) and
// solves the boundary system, phase C recomputes the tile from its carries.
// =========================================================================================
template <typename T, int M, int KY, class Op>
__device__ __forceinline__ void col_chunk(const LineParams<T>& lp, const Op& op, int line, int start,
                                          int cnt, T (&JL)[Op::NF][KY], T (&JR)[Op::NF][KY]) {
    constexpr int NF = Op::NF;
    constexpr int H = M / 2;
    const bool periodic = lp.bc == BC_PERIODIC;
    const int n = lp.n;
    if (cnt <= 0) {
#pragma unroll
        for (int q = 0; q < NF; ++q)
#pragma unroll
            for (int k = 0; k < KY; ++k) JL[q][k] = JR[q][k] = T(0);
        return;
    }
    T win[NF][KY + M];
#pragma unroll
    for (int i = 0; i < KY + M; ++i) {
        T f[NF];
        op.load(line, fold_pos(start - H + i, n, periodic), f);
#pragma unroll
        for (int q = 0; q < NF; ++q) win[q][i] = f[q];
    }
#pragma unroll
    for (int q = 0; q < NF; ++q) {
        local_integrals<T, M, KY>(lp, start, cnt, win[q],
                                  [&](int p) { T f[NF]; op.load(line, p, f); return f[q]; }, JL[q], JR[q]);
    }
}

// Body of one block (32 x WY threads): tile `tile` of the strip of 32 lines from strip*32.
template <typename T, int M, int KY, int WY, class Op>
__device__ __forceinline__ void cols_agg_body(const LineParams<T>& lp, const Op& op, int nlines, T* aggL, T* aggR,
                                              int tiles, int strip, int tile) {
    constexpr int NF = Op::NF;
    constexpr int R = WY * KY;
    __shared__ T sD[WY][32];
    __shared__ T sL[NF][WY][32];
    __shared__ T sR[NF][WY][32];
    const int lane = threadIdx.x, wy = threadIdx.y;
    const int line = strip * 32 + lane;
    const int start = tile * R + wy * KY;
    int cnt = lp.n - start;
    cnt = cnt < 0 ? 0 : (cnt > KY ? KY : cnt);
    if (line >= nlines) cnt = 0;
    T JL[NF][KY], JR[NF][KY];
    col_chunk<T, M, KY>(lp, op, line, start, cnt, JL, JR);
    T D = T(1);
#pragma unroll
    for (int k = 0; k < KY; ++k)
        if (k < cnt) D *= lp.d;
    sD[wy][lane] = D;
#pragma unroll
    for (int q = 0; q < NF; ++q) {
        T a, b;
        chunk_aggregates<T, KY>(lp.d, cnt, JL[q], JR[q], a, b);
        sL[q][wy][lane] = a;
        sR[q][wy][lane] = b;
    }
    __syncthreads();
    if (wy == 0 && line < nlines) {
#pragma unroll
        for (int q = 0; q < NF; ++q) {
            T a = T(0), b = T(0);
            for (int i = 0; i < WY; ++i) a = fma(a, sD[i][lane], sL[q][i][lane]);
            for (int i = WY - 1; i >= 0; --i) b = fma(b, sD[i][lane], sR[q][i][lane]);
            const size_t o = (static_cast<size_t>(q) * tiles + tile) * nlines + line;
            aggL[o] = a;
            aggR[o] = b;
        }
    }
}

template <typename T, int M, int KY, int WY, class Op>
__global__ void __launch_bounds__(32 * WY)
cols_agg_kernel(const __grid_constant__ LineParams<T> lp, const Op op, int nlines, T* aggL, T* aggR, int tiles) {
    cols_agg_body<T, M, KY, WY, Op>(lp, op, nlines, aggL, aggR, tiles, blockIdx.x, blockIdx.y);
}

// One thread per (field, column): scan the tile segments, solve the boundary system in FP64,
// and write the carry entering each tile (or, for walls, the B value injected at the end node).
// The tile recurrences run in the kernel precision (FP64 throughput on this part is a small
// fraction of FP32), with the decays as products of two constants (full tile, last tile).
template <typename T>
__device__ __forceinline__ void carry_body(const LineParams<T>& lp, int nlines, int nf, int tiles, int R,
                                          const T* __restrict__ aggL, const T* __restrict__ aggR,
                                          T* __restrict__ carL, T* __restrict__ carR, int idx) {
    if (idx >= nlines * nf) return;
    const int q = idx / nlines, line = idx % nlines;
    const int n = lp.n;
    const T nu = lp.nu;
    const int last_rows = n - (tiles - 1) * R;
    const T Dfull = dev_exp(-nu * T(R));
    const T Dlast = dev_exp(-nu * T(last_rows));
    const T einv = dev_exp(nu);           // d^{-1}: shifts a power by one node
    const size_t b0 = static_cast<size_t>(q) * tiles * nlines + line;
    auto dec = [&](int t) { return t == tiles - 1 ? Dlast : Dfull; };
    T E = T(0);
#pragma unroll 8
    for (int t = 0; t < tiles; ++t) E = fma(E, dec(t), aggL[b0 + static_cast<size_t>(t) * nlines]);
    const double IN = static_cast<double>(E);
    E = T(0);
#pragma unroll 8
    for (int t = tiles - 1; t >= 0; --t) E = fma(E, dec(t), aggR[b0 + static_cast<size_t>(t) * nlines]);
    const double I0 = static_cast<double>(E);
    const bool periodic = lp.bc == BC_PERIODIC;
    T XL, XR;
    if (periodic) {
        XL = static_cast<T>(IN * lp.inv1mmu);
        XR = static_cast<T>(I0 * lp.inv1mmu);
    } else {
        XL = static_cast<T>(lp.bAA * I0 + lp.bAB * IN);   // B_a
        XR = static_cast<T>(lp.bBA * I0 + lp.bBB * IN);   // B_b
    }
    // forward: carry entering tile t = E_t + d^{s_t} XL (periodic) or E_t + d^{s_t - 1} B_a
    E = T(0);
    T pw = T(1);                           // d^{s_t}
#pragma unroll 8
    for (int t = 0; t < tiles; ++t) {
        T c;
        if (periodic) c = fma(pw, XL, E);
        else c = (t == 0) ? XL : fma(pw * einv, XL, E);
        carL[b0 + static_cast<size_t>(t) * nlines] = c;
        E = fma(E, dec(t), aggL[b0 + static_cast<size_t>(t) * nlines]);
        pw *= dec(t);
    }
    // backward: carry entering tile t from the right = E_t + d^{n-1-e_t} XR (periodic) or
    // E_t + d^{n-2-e_t} B_b, with e_t the tile's last position
    E = T(0);
    T qw = T(1);                           // d^{n-1-e_t}
#pragma unroll 8
    for (int t = tiles - 1; t >= 0; --t) {
        T c;
        if (periodic) c = fma(qw, XR, E);
        else c = (t == tiles - 1) ? XR : fma(qw * einv, XR, E);
        carR[b0 + static_cast<size_t>(t) * nlines] = c;
        E = fma(E, dec(t), aggR[b0 + static_cast<size_t>(t) * nlines]);
        qw *= dec(t);
    }
}

template <typename T>
__global__ void cols_carry_kernel(const __grid_constant__ LineParams<T> lp, int nlines, int nf, int tiles,
                                  int R, const T* __restrict__ aggL, const T* __restrict__ aggR,
                                  T* __restrict__ carL, T* __restrict__ carR) {
    carry_body<T>(lp, nlines, nf, tiles, R, aggL, aggR, carL, carR, blockIdx.x * blockDim.x + threadIdx.x);
}

// The same carries with each column's tiles split over 8 warps.  Block = 32 columns (lanes) x
// 8 warps of one field; warp w scans tiles [w*tpw, (w+1)*tpw).  The warp segments (decay D,
// aggregate E) compose through shared memory, (D1, E1) then (D2, E2) = (D1 D2, E1 D2 + E2),
// giving each warp the segment entering its tiles and every warp the line totals I_N, I_0 for
// the FP64 boundary solve; each warp then writes the carries of its own tiles.  Coalesced over
// the 32 columns and 8x shorter dependency chains than one thread per column.
template <typename T>
__global__ void __launch_bounds__(256)
cols_carry_split_kernel(const __grid_constant__ LineParams<T> lp, int nlines, int nf, int tiles, int R,
                        const T* __restrict__ aggL, const T* __restrict__ aggR, T* __restrict__ carL,
                        T* __restrict__ carR) {
    constexpr int WS = 8;
    __shared__ T sD[WS][32], sEf[WS][32], sEb[WS][32];
    const int lane = threadIdx.x, wy = threadIdx.y;
    const int strips = (nlines + 31) / 32;
    const int q = blockIdx.x / strips;
    const int line = (blockIdx.x % strips) * 32 + lane;
    const bool live = line < nlines && q < nf;
    const int n = lp.n;
    const T nu = lp.nu;
    const int last_rows = n - (tiles - 1) * R;
    const T Dfull = dev_exp(-nu * T(R));
    const T Dlast = dev_exp(-nu * T(last_rows));
    const T einv = dev_exp(nu);           // d^{-1}: shifts a power by one node
    auto dec = [&](int t) { return t == tiles - 1 ? Dlast : Dfull; };
    const int tpw = (tiles + WS - 1) / WS;
    const int t0 = min(wy * tpw, tiles), t1 = min(t0 + tpw, tiles);
    const size_t b0 = static_cast<size_t>(q) * tiles * nlines + line;
    T D = T(1), Ef = T(0), Eb = T(0);
    if (live) {
        for (int t = t0; t < t1; ++t) {
            Ef = fma(Ef, dec(t), aggL[b0 + static_cast<size_t>(t) * nlines]);
            D *= dec(t);
        }
        for (int t = t1 - 1; t >= t0; --t) Eb = fma(Eb, dec(t), aggR[b0 + static_cast<size_t>(t) * nlines]);
    }
    sD[wy][lane] = D;
    sEf[wy][lane] = Ef;
    sEb[wy][lane] = Eb;
    __syncthreads();
    if (!live) return;
    // forward: segment entering this warp (E_in, decay P_in) and the total I_N
    T IN = T(0), P = T(1), Ein = T(0), Pin = T(1);
#pragma unroll
    for (int w = 0; w < WS; ++w) {
        if (w == wy) {
            Ein = IN;
            Pin = P;
        }
        IN = fma(IN, sD[w][lane], sEf[w][lane]);
        P *= sD[w][lane];
    }
    // backward: from the top, entering this warp from the right, and the total I_0
    T I0 = T(0), Q = T(1), Bin = T(0), Qin = T(1);
#pragma unroll
    for (int w = WS - 1; w >= 0; --w) {
        if (w == wy) {
            Bin = I0;
            Qin = Q;
        }
        I0 = fma(I0, sD[w][lane], sEb[w][lane]);
        Q *= sD[w][lane];
    }
    const bool periodic = lp.bc == BC_PERIODIC;
    T XL, XR;
    if (periodic) {
        XL = static_cast<T>(static_cast<double>(IN) * lp.inv1mmu);
        XR = static_cast<T>(static_cast<double>(I0) * lp.inv1mmu);
    } else {
        XL = static_cast<T>(lp.bAA * static_cast<double>(I0) + lp.bAB * static_cast<double>(IN));   // B_a
        XR = static_cast<T>(lp.bBA * static_cast<double>(I0) + lp.bBB * static_cast<double>(IN));   // B_b
    }
    T E = Ein, pw = Pin;
    for (int t = t0; t < t1; ++t) {
        T c;
        if (periodic) c = fma(pw, XL, E);
        else c = (t == 0) ? XL : fma(pw * einv, XL, E);
        carL[b0 + static_cast<size_t>(t) * nlines] = c;
        E = fma(E, dec(t), aggL[b0 + static_cast<size_t>(t) * nlines]);
        pw *= dec(t);
    }
    E = Bin;
    T qw = Qin;
    for (int t = t1 - 1; t >= t0; --t) {
        T c;
        if (periodic) c = fma(qw, XR, E);
        else c = (t == tiles - 1) ? XR : fma(qw * einv, XR, E);
        carR[b0 + static_cast<size_t>(t) * nlines] = c;
        E = fma(E, dec(t), aggR[b0 + static_cast<size_t>(t) * nlines]);
        qw *= dec(t);
    }
}

template <typename T, int M, int KY, int WY, class Op>
__device__ __forceinline__ void cols_final_body(const LineParams<T>& lp, const Op& op, int nlines, const T* carL,
                                                const T* carR, int tiles, int strip, int tile,
                                                unsigned long long* red_slots) {
    constexpr int NF = Op::NF;
    constexpr int R = WY * KY;
    __shared__ T sD[WY][32];
    __shared__ T sL[NF][WY][32];
    __shared__ T sR[NF][WY][32];
    const int lane = threadIdx.x, wy = threadIdx.y;
    const int line = strip * 32 + lane;
    const int n = lp.n;
    const bool periodic = lp.bc == BC_PERIODIC;
    const int start = tile * R + wy * KY;
    int cnt = n - start;
    cnt = cnt < 0 ? 0 : (cnt > KY ? KY : cnt);
    if (line >= nlines) cnt = 0;
    T JL[NF][KY], JR[NF][KY];
    col_chunk<T, M, KY>(lp, op, line, start, cnt, JL, JR);
    T tcL[NF], tcR[NF];
#pragma unroll
    for (int q = 0; q < NF; ++q) {
        tcL[q] = tcR[q] = T(0);
        if (line < nlines) {
            const size_t o = (static_cast<size_t>(q) * tiles + tile) * nlines + line;
            tcL[q] = carL[o];
            tcR[q] = carR[o];
        }
        if (!periodic) {
            // walls: the carry slot of the end tiles holds B_a / B_b, injected at the end node
            if (tile == 0) {
                if (start == 0 && cnt > 0) JL[q][0] += tcL[q];
                tcL[q] = T(0);
            }
            if (tile == tiles - 1) {
#pragma unroll
                for (int k = 0; k < KY; ++k)
                    if (cnt > 0 && k == cnt - 1 && start + k == n - 1) JR[q][k] += tcR[q];
                tcR[q] = T(0);
            }
        }
    }
    T D = T(1);
#pragma unroll
    for (int k = 0; k < KY; ++k)
        if (k < cnt) D *= lp.d;
    sD[wy][lane] = D;
    T aL[NF], aR[NF];
#pragma unroll
    for (int q = 0; q < NF; ++q) {
        chunk_aggregates<T, KY>(lp.d, cnt, JL[q], JR[q], aL[q], aR[q]);
        sL[q][wy][lane] = aL[q];
        sR[q][wy][lane] = aR[q];
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < NF; ++q) {
        T cl = tcL[q];
        for (int i = 0; i < wy; ++i) cl = fma(cl, sD[i][lane], sL[q][i][lane]);
        T cr = tcR[q];
        for (int i = WY - 1; i > wy; --i) cr = fma(cr, sD[i][lane], sR[q][i][lane]);
        chunk_finish<T, KY>(lp.d, cnt, cl, cr, JL[q], JR[q]);
    }
    RedAcc<T> red{T(0), T(0)};
    T aux[KY][Op::NA];
#pragma unroll
    for (int k = 0; k < KY; ++k)
        if (k < cnt) op.fetch(line, start + k, aux[k]);
#pragma unroll
    for (int k = 0; k < KY; ++k) {
        if (k < cnt) {
            T h[NF];
#pragma unroll
            for (int q = 0; q < NF; ++q) h[q] = JR[q][k];
            op.put(line, start + k, h, aux[k], red);
        }
    }
    if (Op::kReduce) block_reduce_store<T>(red, red_slots);
}

template <typename T, int M, int KY, int WY, class Op>
__global__ void __launch_bounds__(32 * WY)
cols_final_kernel(const __grid_constant__ LineParams<T> lp, const Op op, int nlines, const T* carL,
                  const T* carR, int tiles, unsigned long long* red_slots) {
    cols_final_body<T, M, KY, WY, Op>(lp, op, nlines, carL, carR, tiles, blockIdx.x, blockIdx.y, red_slots);
}

}  // namespace molt
