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
template <typename T, int M, int K, class Op>
__global__ void __launch_bounds__(1024)
rows_kernel(const __grid_constant__ LineParams<T> lp, const Op op, int nlines, int tl_log2, int lpb,
            int pitch, unsigned long long* red_slots) {
    constexpr int NF = Op::NF;
    constexpr int H = M / 2;
    extern __shared__ __align__(16) unsigned char smraw[];
    T* sm = reinterpret_cast<T*>(smraw);
    __shared__ T s_scan[32][2 + 2 * NF];   // per-warp segments: D_f, D_b, A_f[NF], A_b[NF]
    __shared__ T s_tot[32][2 * NF];        // per-line totals (lines spanning several warps)
    __shared__ T s_bnd[128][2 * NF];       // per-line carries / B values from the FP64 solve

    const int n = lp.n;
    const bool periodic = lp.bc == BC_PERIODIC;
    const int TL = 1 << tl_log2;
    const int tid = threadIdx.x;
    const int lib = tid >> tl_log2;
    const int t = tid & (TL - 1);
    const int line0 = blockIdx.x * lpb;

    // ---- stage the block's lines (prologue) ----
    for (int l = 0; l < lpb; ++l) {
        const int gl = line0 + l;
        if (gl >= nlines) break;
        T* dst = sm + static_cast<size_t>(l) * NF * pitch;
        for (int p = tid; p < n; p += blockDim.x) {
            T f[NF];
            op.load(gl, p, f);
#pragma unroll
            for (int q = 0; q < NF; ++q) dst[q * pitch + p + (p >> 5)] = f[q];
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
        for (int p = tid; p < n; p += blockDim.x) {
            T h[NF];
#pragma unroll
            for (int q = 0; q < NF; ++q) h[q] = src[q * pitch + p + (p >> 5)];
            op.store(gl, p, h, red);
        }
    }
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

template <typename T, int M, int KY, int WY, class Op>
__global__ void __launch_bounds__(32 * WY)
cols_agg_kernel(const __grid_constant__ LineParams<T> lp, const Op op, int nlines, T* aggL, T* aggR, int tiles) {
    constexpr int NF = Op::NF;
    constexpr int R = WY * KY;
    __shared__ T sD[WY][32];
    __shared__ T sL[NF][WY][32];
    __shared__ T sR[NF][WY][32];
    const int lane = threadIdx.x, wy = threadIdx.y;
    const int line = blockIdx.x * 32 + lane;
    const int tile = blockIdx.y;
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

// One thread per (field, column): scan the tile segments in FP64, solve the boundary system,
// write the carry entering each tile (or, for walls, the B value injected at the end node).
// Decays are products of two constants (full tile, last tile), never per-tile exponentials.
template <typename T>
__global__ void cols_carry_kernel(const __grid_constant__ LineParams<T> lp, int nlines, int nf, int tiles,
                                  int R, const T* aggL, const T* aggR, T* carL, T* carR) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nlines * nf) return;
    const int q = idx / nlines, line = idx % nlines;
    const int n = lp.n;
    const double nu = static_cast<double>(lp.nu);
    const int last_rows = n - (tiles - 1) * R;
    const double Dfull = exp(-nu * R);
    const double Dlast = exp(-nu * last_rows);
    const double einv = exp(nu);          // d^{-1}: shifts a power by one node
    const size_t b0 = static_cast<size_t>(q) * tiles * nlines + line;
    auto dec = [&](int t) { return t == tiles - 1 ? Dlast : Dfull; };
    double E = 0.0;
    for (int t = 0; t < tiles; ++t) E = E * dec(t) + static_cast<double>(aggL[b0 + static_cast<size_t>(t) * nlines]);
    const double IN = E;
    E = 0.0;
    for (int t = tiles - 1; t >= 0; --t) E = E * dec(t) + static_cast<double>(aggR[b0 + static_cast<size_t>(t) * nlines]);
    const double I0 = E;
    const bool periodic = lp.bc == BC_PERIODIC;
    double XL, XR;
    if (periodic) {
        XL = IN * lp.inv1mmu;
        XR = I0 * lp.inv1mmu;
    } else {
        XL = lp.bAA * I0 + lp.bAB * IN;   // B_a
        XR = lp.bBA * I0 + lp.bBB * IN;   // B_b
    }
    // forward: carry entering tile t = E_t + d^{s_t} XL (periodic) or E_t + d^{s_t - 1} B_a
    E = 0.0;
    double pw = 1.0;                        // d^{s_t}
    for (int t = 0; t < tiles; ++t) {
        double c;
        if (periodic) c = E + pw * XL;
        else c = (t == 0) ? XL : E + pw * einv * XL;
        carL[b0 + static_cast<size_t>(t) * nlines] = static_cast<T>(c);
        E = E * dec(t) + static_cast<double>(aggL[b0 + static_cast<size_t>(t) * nlines]);
        pw *= dec(t);
    }
    // backward: carry entering tile t from the right = E_t + d^{n-1-e_t} XR (periodic) or
    // E_t + d^{n-2-e_t} B_b, with e_t the tile's last position
    E = 0.0;
    double qw = 1.0;                        // d^{n-1-e_t}
    for (int t = tiles - 1; t >= 0; --t) {
        double c;
        if (periodic) c = E + qw * XR;
        else c = (t == tiles - 1) ? XR : E + qw * einv * XR;
        carR[b0 + static_cast<size_t>(t) * nlines] = static_cast<T>(c);
        E = E * dec(t) + static_cast<double>(aggR[b0 + static_cast<size_t>(t) * nlines]);
        qw *= dec(t);
    }
}

template <typename T, int M, int KY, int WY, class Op>
__global__ void __launch_bounds__(32 * WY)
cols_final_kernel(const __grid_constant__ LineParams<T> lp, const Op op, int nlines, const T* carL,
                  const T* carR, int tiles, unsigned long long* red_slots) {
    constexpr int NF = Op::NF;
    constexpr int R = WY * KY;
    __shared__ T sD[WY][32];
    __shared__ T sL[NF][WY][32];
    __shared__ T sR[NF][WY][32];
    const int lane = threadIdx.x, wy = threadIdx.y;
    const int line = blockIdx.x * 32 + lane;
    const int tile = blockIdx.y;
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
#pragma unroll
    for (int k = 0; k < KY; ++k) {
        if (k < cnt) {
            T h[NF];
#pragma unroll
            for (int q = 0; q < NF; ++q) h[q] = JR[q][k];
            op.store(line, start + k, h, red);
        }
    }
    if (Op::kReduce) block_reduce_store<T>(red, red_slots);
}

}  // namespace molt
