// Device building blocks of the Helmholtz line sweeps (Sec. 3.2) and the fused per-point
// work of the fixed-point iteration (Sec. 3.1.2, Sec. 5.1).
//
// A thread owns K consecutive positions of one line.  For them it forms the local
// quadrature integrals J^L_j, J^R_j from an (M+1)-point stencil, runs the two exponential
// recurrences of Eq. IL / IR with zero start, and reduces its chunk to a segment
// (D, A): decay over the chunk and recurrence value at the chunk's far end.  Segments
// compose associatively, (D1, A1) then (D2, A2) = (D1 D2, A1 D2 + A2), so a scan over the
// threads of a line gives each chunk the recurrence value entering it; the line totals give
// I_0 and I_N for the boundary 2x2 solve, done in FP64.  A second pass over the chunk, started
// from those carries, produces out_j = I^L_j + B_a d^j + I^R_j + B_b d^{N-j}.
#pragma once

#include <cuda_runtime.h>

#include "molt_internal.h"

namespace molt {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ float dev_exp(float x) { return expf(x); }
__device__ __forceinline__ double dev_exp(double x) { return exp(x); }

// ---- packed FP32 pairs: two fields of one node in one 64-bit register pair, so a stencil or
// recurrence step of both is one fma.rn.f32x2 (each half rounds exactly like fmaf) ----
template <int NF> struct Lanes;
template <> struct Lanes<1> {
    using V = float;
    using W = float;
    static __device__ __forceinline__ V splat(float a) { return a; }
    static __device__ __forceinline__ V fma(V a, V b, V c) { return fmaf(a, b, c); }
    static __device__ __forceinline__ V add(V a, V b) { return a + b; }
    static __device__ __forceinline__ V zero() { return 0.0f; }
    static __device__ __forceinline__ float get(V v, int) { return v; }
    template <int K> static __device__ __forceinline__ V make(const float (&f)[K]) { return f[0]; }
};
template <> struct Lanes<2> {
    using V = unsigned long long;   // low half: field 0, high half: field 1
    using W = unsigned long long;
    static __device__ __forceinline__ V pack(float lo, float hi) {
        V r;
        asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
        return r;
    }
    static __device__ __forceinline__ V splat(float a) { return pack(a, a); }
    static __device__ __forceinline__ V fma(V a, V b, V c) {
        V r;
        asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
        return r;
    }
    static __device__ __forceinline__ V add(V a, V b) {
        V r;
        asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
        return r;
    }
    static __device__ __forceinline__ V zero() { return 0ull; }
    static __device__ __forceinline__ float get(V v, int q) {
        float lo, hi;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
        return q ? hi : lo;
    }
    template <int K> static __device__ __forceinline__ V make(const float (&f)[K]) { return pack(f[0], f[1]); }
};

// Interior stencil weights duplicated into both halves of a 64-bit word (host-built).
struct PackedStencil {
    unsigned long long wl[kMaxStencil];
    unsigned long long wr[kMaxStencil];
};

// Wrap (periodic) or clamp (walls) a position that may lie up to 2n outside the line.
__device__ __forceinline__ int fold_pos(int p, int n, bool periodic) {
    if (periodic) {
        if (p < 0) p += n;
        if (p < 0) p += n;
        if (p >= n) p -= n;
        if (p >= n) p -= n;
        return p;
    }
    return p < 0 ? 0 : (p >= n ? n - 1 : p);
}

// J^L, J^R for positions start..start+K-1 (entries past cnt are left as computed and never
// used).  `win[i]` holds the value at position start - M/2 + i.  `at(p)` returns the value at
// absolute position p; it is only called by the few threads whose chunk touches a wall of a
// non-periodic line (shifted wall stencils, Sec. 3.2 reading).
template <typename T, int M, int K, class At>
__device__ __forceinline__ void local_integrals(const LineParams<T>& lp, int start, int cnt,
                                                const T (&win)[K + M], At at, T (&JL)[K],
                                                T (&JR)[K]) {
    constexpr int H = M / 2;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        T jl = T(0), jr = T(0);
#pragma unroll
        for (int o = 0; o <= M; ++o) {
            jl = fma(lp.wl[o], win[k + o], jl);
            jr = fma(lp.wr[o], win[k + o], jr);
        }
        JL[k] = jl;
        JR[k] = jr;
    }
    if (lp.bc != BC_PERIODIC) {
        const int N = lp.N;
        const int jb = N - H + 1;
        if (start < H || start + cnt - 1 >= jb) {
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const int j = start + k;
                if (k >= cnt) continue;
                if (j < H) {
                    T jl = T(0), jr = T(0);
                    for (int o = 0; o <= M; ++o) {
                        const T v = at(o);
                        if (j >= 1) jl = fma(lp.wlA[j - 1][o], v, jl);
                        jr = fma(lp.wrA[j][o], v, jr);
                    }
                    JL[k] = jl;      // J^L_0 = 0: I^L_0 = 0 (Eq. IL)
                    JR[k] = jr;
                } else if (j >= jb) {
                    T jl = T(0), jr = T(0);
                    for (int o = 0; o <= M; ++o) {
                        const T v = at(N - M + o);
                        jl = fma(lp.wlB[j - jb][o], v, jl);
                        if (j < N) jr = fma(lp.wrB[j - jb][o], v, jr);
                    }
                    JL[k] = jl;
                    JR[k] = jr;      // J^R_N = 0: I^R_N = 0 (Eq. IR)
                }
            }
        }
    }
}

// Zero-start recurrences over the chunk: aL = I^L at the chunk's last position,
// aR = I^R at its first position (Eq. IL / IR restricted to the chunk).
template <typename T, int K>
__device__ __forceinline__ void chunk_aggregates(T d, int cnt, const T (&JL)[K], const T (&JR)[K],
                                                 T& aL, T& aR) {
    T a = T(0), b = T(0);
#pragma unroll
    for (int k = 0; k < K; ++k)
        if (k < cnt) a = fma(d, a, JL[k]);
#pragma unroll
    for (int k = K - 1; k >= 0; --k)
        if (k < cnt) b = fma(d, b, JR[k]);
    aL = a;
    aR = b;
}

// Second pass: out_k = P^R_k + P^L_k from the carries entering the chunk from the right (cR)
// and from the left (cL).  The result overwrites JR.
template <typename T, int K>
__device__ __forceinline__ void chunk_finish(T d, int cnt, T cL, T cR, const T (&JL)[K], T (&JR)[K]) {
    T p = cR;
#pragma unroll
    for (int k = K - 1; k >= 0; --k)
        if (k < cnt) {
            p = fma(d, p, JR[k]);
            JR[k] = p;
        }
    T q = cL;
#pragma unroll
    for (int k = 0; k < K; ++k)
        if (k < cnt) {
            q = fma(d, q, JL[k]);
            JR[k] += q;
        }
}

// ---------------------------------------------------------------------------------------
// Per-point work of each pass, fused into the sweeps as load (prologue) / store (epilogue).
// kAxes: 1 = runs on rows (x), 2 = on columns (y), 3 = both.
// A field element of a line is at index line * ls + pos * ps.
// G(x) = x (x (x + g2) + g1) is the lagged nonlinear term in the stored variable x = u
// (= v - 1): G = x^3 + (lam - 3) x, i.e. G(v) without its constant lam - 2.  Under periodic and
// Neumann conditions every operator that constant passes through maps it to zero; under Dirichlet
// conditions its image (with that of the shift) is the separable FP64 offset added to Y once per
// stage (Eq. 2D_Helmholtz applied to constants).  g2 = g1 = 0 selects G = 0 (the linear parts
// of a stage).
// ---------------------------------------------------------------------------------------

// Residual accumulators in the kernel precision: |w_new - w| of two nearby floats is exact
// (Sterbenz), and a max is exact in any precision; the block result is widened to FP64.
template <typename T>
struct RedAcc {
    T dmax;   // max |w_new - w|
    T vmax;   // max |w_new| (stored variable)
};

template <typename T>
struct OpBase {
    long long ls, ps;
    __device__ __forceinline__ size_t at(int line, int pos) const {
        return static_cast<size_t>(line) * static_cast<size_t>(ls) + static_cast<size_t>(pos) * static_cast<size_t>(ps);
    }
};

template <typename T>
__device__ __forceinline__ T g_lag(T x, T g2, T g1) { return x * fma(x, x + g2, g1); }

// Each op: load() = prologue (reads the inputs at a point, returns the NF fields to sweep);
// fetch() = the extra inputs the epilogue needs (NA values, read before any store so that the
// loads of a batch of points are in flight together); put() = epilogue arithmetic and stores.

// H applied to one field.
template <typename T>
struct OpCopy : OpBase<T> {
    static constexpr int NF = 1;
    static constexpr int NA = 1;
    static constexpr int kAxes = 3;
    static constexpr bool kReduce = false;
    const T* in;
    T* out;
    __device__ __forceinline__ void load(int line, int pos, T (&f)[1]) const { f[0] = in[this->at(line, pos)]; }
    __device__ __forceinline__ void fetch(int, int, T (&)[NA]) const {}
    __device__ __forceinline__ void put(int line, int pos, const T (&h)[1], const T (&)[NA], RedAcc<T>&) const {
        out[this->at(line, pos)] = h[0];
    }
};

// 2D pass 1 (y, inner c): T = H_iy G(w), S = H_iy w.
template <typename T>
struct OpP1 : OpBase<T> {
    static constexpr int NF = 2;
    static constexpr int NA = 1;
    static constexpr int kAxes = 2;
    static constexpr bool kReduce = false;
    const T* w;
    T* t_out;
    T* s_out;
    T g2, g1;
    __device__ __forceinline__ void load(int line, int pos, T (&f)[2]) const {
        const T x = w[this->at(line, pos)];
        f[0] = g_lag(x, g2, g1);
        f[1] = x;
    }
    __device__ __forceinline__ void fetch(int, int, T (&)[NA]) const {}
    __device__ __forceinline__ void put(int line, int pos, const T (&h)[2], const T (&)[NA], RedAcc<T>&) const {
        const size_t i = this->at(line, pos);
        t_out[i] = h[0];
        s_out[i] = h[1];
    }
};

// 2D pass 2 (x, inner c): with A1 = H_ix(2T - G), A2 = H_ix(w - S):
//   U = S + A2 (= w - D_ix D_iy w),  P = beta (A1 - T) + U
// (beta (A1 - T) = beta (M_i^{-1} G - G + D_ix D_iy G)).
template <typename T>
struct OpP2 : OpBase<T> {
    static constexpr int NF = 2;
    static constexpr int NA = 2;
    static constexpr int kAxes = 1;
    static constexpr bool kReduce = false;
    const T* w;
    const T* t_in;
    const T* s_in;
    T* p_out;
    T* u_out;
    T g2, g1, beta;
    __device__ __forceinline__ void load(int line, int pos, T (&f)[2]) const {
        const size_t i = this->at(line, pos);
        const T x = w[i];
        f[0] = T(2) * t_in[i] - g_lag(x, g2, g1);
        f[1] = x - s_in[i];
    }
    __device__ __forceinline__ void fetch(int line, int pos, T (&a)[NA]) const {
        const size_t i = this->at(line, pos);
        a[0] = t_in[i];
        a[1] = s_in[i];
    }
    __device__ __forceinline__ void put(int line, int pos, const T (&h)[2], const T (&a)[NA], RedAcc<T>&) const {
        const size_t i = this->at(line, pos);
        const T u = a[1] + h[1];
        u_out[i] = u;
        p_out[i] = fma(beta, h[0] - a[0], u);
    }
};

// 2D pass 3 (y, outer c): Q1 = H_oy P, Q2 = H_oy U.
template <typename T>
struct OpP3 : OpBase<T> {
    static constexpr int NF = 2;
    static constexpr int NA = 1;
    static constexpr int kAxes = 2;
    static constexpr bool kReduce = false;
    const T* p_in;
    const T* u_in;
    T* q1_out;
    T* q2_out;
    __device__ __forceinline__ void load(int line, int pos, T (&f)[2]) const {
        const size_t i = this->at(line, pos);
        f[0] = p_in[i];
        f[1] = u_in[i];
    }
    __device__ __forceinline__ void fetch(int, int, T (&)[NA]) const {}
    __device__ __forceinline__ void put(int line, int pos, const T (&h)[2], const T (&)[NA], RedAcc<T>&) const {
        const size_t i = this->at(line, pos);
        q1_out[i] = h[0];
        q2_out[i] = h[1];
    }
};

// 2D pass 4 (x, outer c): w_new = Y + w - Q2 + H_ox(Q1 - U), written over w, with the
// residual max |w_new - w| and the scale max |w_new|.
template <typename T>
struct OpP4 : OpBase<T> {
    static constexpr int NF = 1;
    static constexpr int NA = 3;
    static constexpr int kAxes = 1;
    static constexpr bool kReduce = true;
    const T* q1_in;
    const T* q2_in;
    const T* u_in;
    const T* y_in;
    T* w;
    T shift;
    __device__ __forceinline__ void load(int line, int pos, T (&f)[1]) const {
        const size_t i = this->at(line, pos);
        f[0] = q1_in[i] - u_in[i];
    }
    __device__ __forceinline__ void fetch(int line, int pos, T (&a)[NA]) const {
        const size_t i = this->at(line, pos);
        a[0] = w[i];
        a[1] = y_in[i];
        a[2] = q2_in[i];
    }
    __device__ __forceinline__ void put(int line, int pos, const T (&h)[1], const T (&a)[NA], RedAcc<T>& r) const {
        const T nw = (a[1] + a[0] - a[2]) + h[0];
        w[this->at(line, pos)] = nw;
        r.dmax = fmax(r.dmax, fabs(nw - a[0]));
        r.vmax = fmax(r.vmax, fabs(nw));
    }
};

// 3D split stage, x lines (rows only): out = H_x[ka (y + z) + kb yz] + kc yz, with y = H_y f,
// z = H_z f and yz = H_y H_z f of one field f.  The pair and triple products of the 3D remainder
// X regroup by linearity of H_x into this one sweep: (ka, kb, kc) = s (1, -2, 1) gives s Q f and
// s (-1, 3, -1) gives s A f.
template <typename T>
struct OpComb3 : OpBase<T> {
    static constexpr int NF = 1;
    static constexpr int NA = 1;
    static constexpr int kAxes = 1;
    static constexpr bool kReduce = false;
    const T* y;
    const T* z;
    const T* yz;
    T* out;
    T ka, kb, kc;
    __device__ __forceinline__ void load(int line, int pos, T (&f)[1]) const {
        const size_t i = this->at(line, pos);
        f[0] = fma(kb, yz[i], ka * (y[i] + z[i]));
    }
    __device__ __forceinline__ void fetch(int line, int pos, T (&a)[NA]) const { a[0] = yz[this->at(line, pos)]; }
    __device__ __forceinline__ void put(int line, int pos, const T (&h)[1], const T (&a)[NA], RedAcc<T>&) const {
        out[this->at(line, pos)] = fma(kc, a[0], h[0]);
    }
};

// 1D pass a (inner c): E = H_i[beta G(w)] - beta G(w).
template <typename T>
struct Op1a : OpBase<T> {
    static constexpr int NF = 1;
    static constexpr int NA = 1;
    static constexpr int kAxes = 1;
    static constexpr bool kReduce = false;
    const T* w;
    T* e_out;
    T g2, g1, beta;
    __device__ __forceinline__ void load(int line, int pos, T (&f)[1]) const {
        f[0] = beta * g_lag(w[this->at(line, pos)], g2, g1);
    }
    __device__ __forceinline__ void fetch(int line, int pos, T (&a)[NA]) const { a[0] = w[this->at(line, pos)]; }
    __device__ __forceinline__ void put(int line, int pos, const T (&h)[1], const T (&a)[NA], RedAcc<T>&) const {
        e_out[this->at(line, pos)] = h[0] - beta * g_lag(a[0], g2, g1);
    }
};

// 1D pass b (outer c): w_new = Y + H_o E over w, with the residual.
template <typename T>
struct Op1b : OpBase<T> {
    static constexpr int NF = 1;
    static constexpr int NA = 2;
    static constexpr int kAxes = 1;
    static constexpr bool kReduce = true;
    const T* e_in;
    const T* y_in;
    T* w;
    T shift;
    __device__ __forceinline__ void load(int line, int pos, T (&f)[1]) const { f[0] = e_in[this->at(line, pos)]; }
    __device__ __forceinline__ void fetch(int line, int pos, T (&a)[NA]) const {
        const size_t i = this->at(line, pos);
        a[0] = w[i];
        a[1] = y_in[i];
    }
    __device__ __forceinline__ void put(int line, int pos, const T (&h)[1], const T (&a)[NA], RedAcc<T>& r) const {
        const T nw = a[1] + h[0];
        w[this->at(line, pos)] = nw;
        r.dmax = fmax(r.dmax, fabs(nw - a[0]));
        r.vmax = fmax(r.vmax, fabs(nw));
    }
};

// ---- Vector CH (Sec. 5.2): two components in the stored variable v = u - z3 ----
// Lagged term of component `comp`: G = [grad W(v + z3)]_comp - s v_comp with
// grad W = 6 (z^3 - 1) conj(z^2), z = u1 + i u2 (W = |z^3 - 1|^2, Eq. CH_vector_reaction), and
// s = (c1 + c2)/tau the linear part the factorization moves to the left (Eq. CH_vector_fixed1/2).
template <typename T>
__device__ __forceinline__ T vch_lag(T v1, T v2, int comp, T s) {
    const T a = v1 - T(0.5), b = v2 - T(0.86602540378443864676);   // u = v + z3
    const T a2 = a * a, b2 = b * b;
    const T fr = a * (a2 - T(3) * b2) - T(1), fi = b * (T(3) * a2 - b2);   // z^3 - 1
    const T zr = a2 - b2, zi = T(2) * a * b;                                // z^2
    return comp == 0 ? T(6) * (fr * zr + fi * zi) - s * v1 : T(6) * (fi * zr - fr * zi) - s * v2;
}

// 2D pass 1 of component comp (y, inner c): T = H_iy G_comp(v), S = H_iy v_comp.
template <typename T>
struct OpP1V : OpBase<T> {
    static constexpr int NF = 2;
    static constexpr int NA = 1;
    static constexpr int kAxes = 2;
    static constexpr bool kReduce = false;
    const T* v1;
    const T* v2;
    T* t_out;
    T* s_out;
    T s;
    int comp;
    __device__ __forceinline__ void load(int line, int pos, T (&f)[2]) const {
        const size_t i = this->at(line, pos);
        const T x1 = v1[i], x2 = v2[i];
        f[0] = vch_lag(x1, x2, comp, s);
        f[1] = comp == 0 ? x1 : x2;
    }
    __device__ __forceinline__ void fetch(int, int, T (&)[NA]) const {}
    __device__ __forceinline__ void put(int line, int pos, const T (&h)[2], const T (&)[NA], RedAcc<T>&) const {
        const size_t i = this->at(line, pos);
        t_out[i] = h[0];
        s_out[i] = h[1];
    }
};

// 2D pass 2 of component comp (x, inner c): OpP2 with G_comp(v) in place of G(w).
template <typename T>
struct OpP2V : OpBase<T> {
    static constexpr int NF = 2;
    static constexpr int NA = 2;
    static constexpr int kAxes = 1;
    static constexpr bool kReduce = false;
    const T* v1;
    const T* v2;
    const T* t_in;
    const T* s_in;
    T* p_out;
    T* u_out;
    T s, beta;
    int comp;
    __device__ __forceinline__ void load(int line, int pos, T (&f)[2]) const {
        const size_t i = this->at(line, pos);
        const T x1 = v1[i], x2 = v2[i];
        f[0] = T(2) * t_in[i] - vch_lag(x1, x2, comp, s);
        f[1] = (comp == 0 ? x1 : x2) - s_in[i];
    }
    __device__ __forceinline__ void fetch(int line, int pos, T (&a)[NA]) const {
        const size_t i = this->at(line, pos);
        a[0] = t_in[i];
        a[1] = s_in[i];
    }
    __device__ __forceinline__ void put(int line, int pos, const T (&h)[2], const T (&a)[NA], RedAcc<T>&) const {
        const size_t i = this->at(line, pos);
        const T u = a[1] + h[1];
        u_out[i] = u;
        p_out[i] = fma(beta, h[0] - a[0], u);
    }
};

// 1D pass a of component comp (inner c): E = H_i[beta G_comp(v)] - beta G_comp(v).
template <typename T>
struct Op1aV : OpBase<T> {
    static constexpr int NF = 1;
    static constexpr int NA = 2;
    static constexpr int kAxes = 1;
    static constexpr bool kReduce = false;
    const T* v1;
    const T* v2;
    T* e_out;
    T s, beta;
    int comp;
    __device__ __forceinline__ void load(int line, int pos, T (&f)[1]) const {
        const size_t i = this->at(line, pos);
        f[0] = beta * vch_lag(v1[i], v2[i], comp, s);
    }
    __device__ __forceinline__ void fetch(int line, int pos, T (&a)[NA]) const {
        const size_t i = this->at(line, pos);
        a[0] = v1[i];
        a[1] = v2[i];
    }
    __device__ __forceinline__ void put(int line, int pos, const T (&h)[1], const T (&a)[NA], RedAcc<T>&) const {
        e_out[this->at(line, pos)] = h[0] - beta * vch_lag(a[0], a[1], comp, s);
    }
};

// Block-wide max of the two residual values, then one atomic max per block on the
// bit patterns (non-negative doubles order like their unsigned bits).
template <typename T>
__device__ __forceinline__ void block_reduce_store(RedAcc<T> r, unsigned long long* slots) {
    __shared__ double s_d[32], s_v[32];
    double a = static_cast<double>(r.dmax), b = static_cast<double>(r.vmax);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a = fmax(a, __shfl_xor_sync(kFull, a, o));
        b = fmax(b, __shfl_xor_sync(kFull, b, o));
    }
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int nthreads = blockDim.x * blockDim.y;
    const int warp = tid >> 5, lane = tid & 31;
    if (lane == 0) {
        s_d[warp] = a;
        s_v[warp] = b;
    }
    __syncthreads();
    if (warp == 0) {
        const int nw = (nthreads + 31) >> 5;
        a = lane < nw ? s_d[lane] : 0.0;
        b = lane < nw ? s_v[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a = fmax(a, __shfl_xor_sync(kFull, a, o));
            b = fmax(b, __shfl_xor_sync(kFull, b, o));
        }
        if (lane == 0) {
            atomicMax(&slots[0], static_cast<unsigned long long>(__double_as_longlong(a)));
            atomicMax(&slots[1], static_cast<unsigned long long>(__double_as_longlong(b)));
        }
    }
}

}  // namespace molt

namespace molt {

// ---------------------------------------------------------------------------------------
// Pointwise forms of the row passes for the pipelined FP32 row kernel: NS fields are staged
// (double-buffered in shared memory), NA auxiliary fields are prefetched for the epilogue,
// NO outputs are written.  prologue(): staged values -> fields to sweep; epilogue(): swept
// values + staged + auxiliary -> outputs.
// ---------------------------------------------------------------------------------------
template <typename T>
struct PipeCopy {
    static constexpr int NS = 1, NA = 0, NF = 1, NO = 1;
    static constexpr bool kReduce = false;
    const T* s[NS];
    const T* a[1];
    T* o[NO];
    T g2, g1, beta;
    __device__ __forceinline__ void prologue(const T (&sv)[NS], T (&f)[NF]) const { f[0] = sv[0]; }
    __device__ __forceinline__ void epilogue(const T (&h)[NF], const T (&)[NS], const T (&)[1], T (&ov)[NO],
                                             RedAcc<T>&) const { ov[0] = h[0]; }
};

// pass 2 (x, inner c): staged w, T, S; outputs P, U (see OpP2)
template <typename T>
struct PipeP2 {
    static constexpr int NS = 3, NA = 0, NF = 2, NO = 2;
    static constexpr bool kReduce = false;
    const T* s[NS];
    const T* a[1];
    T* o[NO];
    T g2, g1, beta;
    __device__ __forceinline__ void prologue(const T (&sv)[NS], T (&f)[NF]) const {
        f[0] = T(2) * sv[1] - g_lag(sv[0], g2, g1);
        f[1] = sv[0] - sv[2];
    }
    __device__ __forceinline__ void epilogue(const T (&h)[NF], const T (&sv)[NS], const T (&)[1], T (&ov)[NO],
                                             RedAcc<T>&) const {
        const T u = sv[2] + h[1];
        ov[0] = fma(beta, h[0] - sv[1], u);
        ov[1] = u;
    }
};

// 3D x lines: staged y, z, yz; output H[ka (y + z) + kb yz] + kc yz (see OpComb3; ka = g2,
// kb = g1, kc = beta)
template <typename T>
struct PipeComb3 {
    static constexpr int NS = 3, NA = 0, NF = 1, NO = 1;
    static constexpr bool kReduce = false;
    const T* s[NS];
    const T* a[1];
    T* o[NO];
    T g2, g1, beta;
    __device__ __forceinline__ void prologue(const T (&sv)[NS], T (&f)[NF]) const {
        f[0] = fma(g1, sv[2], g2 * (sv[0] + sv[1]));
    }
    __device__ __forceinline__ void epilogue(const T (&h)[NF], const T (&sv)[NS], const T (&)[1], T (&ov)[NO],
                                             RedAcc<T>&) const {
        ov[0] = fma(beta, sv[2], h[0]);
    }
};

// pass 4 (x, outer c): staged Q1, U; auxiliary w, Y, Q2; output w_new (over w)
template <typename T>
struct PipeP4 {
    static constexpr int NS = 2, NA = 3, NF = 1, NO = 1;
    static constexpr bool kReduce = true;
    const T* s[NS];
    const T* a[NA];
    T* o[NO];
    T g2, g1, beta;
    __device__ __forceinline__ void prologue(const T (&sv)[NS], T (&f)[NF]) const { f[0] = sv[0] - sv[1]; }
    __device__ __forceinline__ void epilogue(const T (&h)[NF], const T (&)[NS], const T (&av)[NA], T (&ov)[NO],
                                             RedAcc<T>& r) const {
        const T nw = (av[1] + av[0] - av[2]) + h[0];
        ov[0] = nw;
        r.dmax = fmax(r.dmax, fabs(nw - av[0]));
        r.vmax = fmax(r.vmax, fabs(nw));
    }
};

// 1D pass a: staged w; output E = H_i[beta G(w)] - beta G(w)
template <typename T>
struct Pipe1a {
    static constexpr int NS = 1, NA = 0, NF = 1, NO = 1;
    static constexpr bool kReduce = false;
    const T* s[NS];
    const T* a[1];
    T* o[NO];
    T g2, g1, beta;
    __device__ __forceinline__ void prologue(const T (&sv)[NS], T (&f)[NF]) const {
        f[0] = beta * g_lag(sv[0], g2, g1);
    }
    __device__ __forceinline__ void epilogue(const T (&h)[NF], const T (&sv)[NS], const T (&)[1], T (&ov)[NO],
                                             RedAcc<T>&) const {
        ov[0] = h[0] - beta * g_lag(sv[0], g2, g1);
    }
};

// 1D pass b: staged E; auxiliary w, Y; output w_new = Y + H_o E (over w)
template <typename T>
struct Pipe1b {
    static constexpr int NS = 1, NA = 2, NF = 1, NO = 1;
    static constexpr bool kReduce = true;
    const T* s[NS];
    const T* a[NA];
    T* o[NO];
    T g2, g1, beta;
    __device__ __forceinline__ void prologue(const T (&sv)[NS], T (&f)[NF]) const { f[0] = sv[0]; }
    __device__ __forceinline__ void epilogue(const T (&h)[NF], const T (&)[NS], const T (&av)[NA], T (&ov)[NO],
                                             RedAcc<T>& r) const {
        const T nw = av[1] + h[0];
        ov[0] = nw;
        r.dmax = fmax(r.dmax, fabs(nw - av[0]));
        r.vmax = fmax(r.vmax, fabs(nw));
    }
};

// vector CH pass 2 of component comp: staged v1, v2, T, S; outputs P, U (see OpP2V)
template <typename T>
struct PipeP2V {
    static constexpr int NS = 4, NA = 0, NF = 2, NO = 2;
    static constexpr bool kReduce = false;
    const T* s[NS];
    const T* a[1];
    T* o[NO];
    T g2, g1, beta;
    T vs;
    int comp;
    __device__ __forceinline__ void prologue(const T (&sv)[NS], T (&f)[NF]) const {
        f[0] = T(2) * sv[2] - vch_lag(sv[0], sv[1], comp, vs);
        f[1] = (comp == 0 ? sv[0] : sv[1]) - sv[3];
    }
    __device__ __forceinline__ void epilogue(const T (&h)[NF], const T (&sv)[NS], const T (&)[1], T (&ov)[NO],
                                             RedAcc<T>&) const {
        const T u = sv[3] + h[1];
        ov[0] = fma(beta, h[0] - sv[2], u);
        ov[1] = u;
    }
};

// vector CH 1D pass a of component comp: staged v1, v2; output E (see Op1aV)
template <typename T>
struct Pipe1aV {
    static constexpr int NS = 2, NA = 0, NF = 1, NO = 1;
    static constexpr bool kReduce = false;
    const T* s[NS];
    const T* a[1];
    T* o[NO];
    T g2, g1, beta;
    T vs;
    int comp;
    __device__ __forceinline__ void prologue(const T (&sv)[NS], T (&f)[NF]) const {
        f[0] = beta * vch_lag(sv[0], sv[1], comp, vs);
    }
    __device__ __forceinline__ void epilogue(const T (&h)[NF], const T (&sv)[NS], const T (&)[1], T (&ov)[NO],
                                             RedAcc<T>&) const {
        ov[0] = h[0] - beta * vch_lag(sv[0], sv[1], comp, vs);
    }
};

// Ampere-style asynchronous 16-byte global -> shared copies (LDGSTS), grouped and awaited.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// 16-byte chunk swizzle inside each 128-byte group of 8 chunks: chunk c lives at
// c ^ ((c >> 3) & 7).  With 4 (or 2) chunks per thread the 8 lanes of each 128-bit
// shared access phase hit 8 distinct bank groups.
__device__ __forceinline__ int swz(int c) { return c ^ ((c >> 3) & 7); }

}  // namespace molt

namespace molt {

// Column passes in pointwise form (pipelined FP32 column kernels).
// pass 1 (y, inner c): staged w; sweep G(w), w; outputs T = H G, S = H w
template <typename T>
struct PipeP1 {
    static constexpr int NS = 1, NA = 0, NF = 2, NO = 2;
    static constexpr bool kReduce = false;
    const T* s[NS];
    const T* a[1];
    T* o[NO];
    T g2, g1, beta;
    __device__ __forceinline__ void prologue(const T (&sv)[NS], T (&f)[NF]) const {
        f[0] = g_lag(sv[0], g2, g1);
        f[1] = sv[0];
    }
    __device__ __forceinline__ void epilogue(const T (&h)[NF], const T (&)[NS], const T (&)[1], T (&ov)[NO],
                                             RedAcc<T>&) const {
        ov[0] = h[0];
        ov[1] = h[1];
    }
};

// vector CH pass 1 of component comp (y, inner c): staged v1, v2; sweep G_comp(v), v_comp;
// outputs T, S (see OpP1V)
template <typename T>
struct PipeP1V {
    static constexpr int NS = 2, NA = 0, NF = 2, NO = 2;
    static constexpr bool kReduce = false;
    const T* s[NS];
    const T* a[1];
    T* o[NO];
    T g2, g1, beta;
    T vs;
    int comp;
    __device__ __forceinline__ void prologue(const T (&sv)[NS], T (&f)[NF]) const {
        f[0] = vch_lag(sv[0], sv[1], comp, vs);
        f[1] = comp == 0 ? sv[0] : sv[1];
    }
    __device__ __forceinline__ void epilogue(const T (&h)[NF], const T (&)[NS], const T (&)[1], T (&ov)[NO],
                                             RedAcc<T>&) const {
        ov[0] = h[0];
        ov[1] = h[1];
    }
};

// pass 3 (y, outer c): staged P, U; outputs Q1 = H P, Q2 = H U
template <typename T>
struct PipeP3 {
    static constexpr int NS = 2, NA = 0, NF = 2, NO = 2;
    static constexpr bool kReduce = false;
    const T* s[NS];
    const T* a[1];
    T* o[NO];
    T g2, g1, beta;
    __device__ __forceinline__ void prologue(const T (&sv)[NS], T (&f)[NF]) const {
        f[0] = sv[0];
        f[1] = sv[1];
    }
    __device__ __forceinline__ void epilogue(const T (&h)[NF], const T (&)[NS], const T (&)[1], T (&ov)[NO],
                                             RedAcc<T>&) const {
        ov[0] = h[0];
        ov[1] = h[1];
    }
};

}  // namespace molt
