// C ABI of the library (include/molt.h): handles, stage solves and time schemes.
//
// Stored variable.  The kernels work on w = v - 1 = u with v = u + 1 (Sec. 3), so the constant
// part of v never passes through FP32 arithmetic and every field is rounded relative to |u|, not
// |v|.  On periodic and Neumann grids every line inverse maps constants to themselves, so the
// fixed-point map keeps the same form in w: D = I - H annihilates constants and all right-hand-side
// combinations below have coefficients summing to one.  Dirichlet inverses hold v = 0 on the
// walls and do not map 1 to itself; there the constant part adds one fixed field per stage
// coefficient to Y (add_dirichlet_offset), and the iteration is otherwise the same.
//
// Stage solve (v - tau F(v) = r):  parameters from the regime switch of Sec. 3.1.2 (with
// dt -> tau as in Sec. 4.1-4.2), inner factor = larger c.
//   1D:  w <- H_o[ H_i[r + beta G(w)] - beta G(w) ]                     (2 sweeps)
//   2D:  Y = H_ox H_oy H_ix H_iy r once, then per iteration
//        (y, c_i)  T = H_iy G(w),  S = H_iy w
//        (x, c_i)  U = S + H_ix(w - S),  P = beta (H_ix(2T - G) - T) + U
//        (y, c_o)  Q1 = H_oy P,  Q2 = H_oy U
//        (x, c_o)  w <- Y + w - Q2 + H_ox(Q1 - U)
//   which is, term by term, Y + M_o^{-1}[beta (M_i^{-1}G - G + D_ix D_iy G)]
//   + (D_ox D_oy + D_ix D_iy - D_ox D_oy D_ix D_iy) w  (Sec. 5.1 with c_o != c_i).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/molt.h"
#include "molt_internal.h"

struct molt_grid {
    int dim, nx, ny;
    double Lx, Ly;
    int bc;
};

namespace {

thread_local std::string g_last_error = "";
std::atomic<long long> g_tma_launches{0};

constexpr double kEta2 = 0.29289321881345247560;   // 1 - sqrt(2)/2 (Sec. 4.2)

double alexander_eta() {
    // root of x^3 - 3x^2 + 3x/2 - 1/6 in (0.4, 0.5): Alexander's L-stable SDIRK3 (Sec. 4.4 quotes 0.4359)
    double lo = 0.4, hi = 0.5;
    auto p = [](double x) { return ((x - 3.0) * x + 1.5) * x - 1.0 / 6.0; };
    for (int i = 0; i < 200; ++i) {
        const double mid = 0.5 * (lo + hi);
        if (p(lo) * p(mid) <= 0) hi = mid;
        else lo = mid;
    }
    return 0.5 * (lo + hi);
}

}  // namespace

molt::StageParams molt::stage_params(double tau, double eps) {
    StageParams sp;
    double c1, c2;
    if (tau >= eps * eps) {
        const double disc = std::sqrt(tau * tau - eps * eps * tau);
        c1 = tau + disc;
        c2 = tau - disc;
        sp.factor = true;
    } else {
        c1 = c2 = std::sqrt(eps * eps * tau);
        sp.factor = false;
    }
    sp.c_in = std::max(c1, c2);
    sp.c_out = std::min(c1, c2);
    sp.beta = tau / sp.c_in;
    sp.lam = 2.0 - (c1 + c2) / tau;
    return sp;
}

double molt::grid_h(int n, double L, int bc) { return bc == molt::BC_PERIODIC ? L / n : L / (n - 1); }

// Dirichlet offset of a stage (see the file comment).  With K the fused passes in w and K_v the same
// passes in v (where G(1) = lambda - 2 =: g0),
//   w_new = v_new - 1 = [Y_w + M_o^{-1} M_i^{-1} 1 + K_v(1) - 1] + K(w),
// and the bracket's fixed part C is a sum of products of line profiles, from the passes applied to
// v = 1 (T = g0 phi_iy, S = phi_iy, U, P, Q1, Q2 with phi_a = H_a 1):
//   2D: C = psi1 (psi2 + H_oy p1 - a2) - phi_ix H_oy a2 + phi_ox (H_oy p0 - phi_iy) - psi2,
//       a2 = 1 - phi_iy, p1 = (2 beta g0 - 1) phi_iy + 1 - beta g0, p0 = (1 - beta g0) phi_iy,
//       psi1 = H_ox phi_ix, psi2 = H_oy phi_iy;
//   1D: C = (1 + beta g0) psi1 - beta g0 phi_o - 1, psi1 = H_o phi_i.
// C vanishes away from the walls (all profiles -> 1).  The profiles are FP64 sweeps of single lines
// into `prof` (kOffsetProfiles rows of L >= max(nx, ny) doubles); *out receives the products.
cudaError_t molt::dirichlet_offset(const LineParams<double> lp[4], int dim, double bg, double* prof, int L,
                                   Separable* out, cudaStream_t st, long long* launches) {
    auto P = [&](int k) { return prof + static_cast<size_t>(k) * L; };
    auto sweep1 = [&](const LineParams<double>& l, const double* in, double* o) {
        OpArgs<double> a;
        a.in0 = in;
        a.out0 = o;
        return molt::sweep<double>(0, l, OP_COPY, a, l.n, 1, nullptr, nullptr, st, launches, nullptr);
    };
    auto lin1 = [&](double* o, int n, const double* x0, double c0, const double* x1, double c1, double c4) {
        return molt::lincomb<double>(o, n, x0, c0, x1, c1, nullptr, 0, nullptr, 0, c4, st, launches);
    };
    const LineParams<double>&lix = lp[0], &lox = lp[1];
    const int nx = lix.n;
    cudaError_t e;
    // x profiles: 0 = 1, 1 = phi_ix, 2 = phi_ox, 3 = psi1
    if ((e = lin1(P(0), nx, nullptr, 0, nullptr, 0, 1.0)) != cudaSuccess || (e = sweep1(lix, P(0), P(1))) != cudaSuccess ||
        (e = sweep1(lox, P(0), P(2))) != cudaSuccess || (e = sweep1(lox, P(1), P(3))) != cudaSuccess)
        return e;
    if (dim == 1) {
        // beta_0 = (1 + beta g0) psi1 - beta g0 phi_o - 1 in profile 4, alpha_0 = 1 (profile 0)
        if ((e = lin1(P(4), nx, P(3), 1.0 + bg, P(2), -bg, -1.0)) != cudaSuccess) return e;
        *out = Separable{{P(0)}, {P(4)}, 1};
        return cudaSuccess;
    }
    const LineParams<double>&liy = lp[2], &loy = lp[3];
    const int ny = liy.n;
    // y profiles: 5 = 1, 6 = phi_iy, 7 = a2, 8 = p1, 9 = p0, 10 = psi2, 11 = H_oy a2, 12 = H_oy p1,
    // 13 = H_oy p0
    if ((e = lin1(P(5), ny, nullptr, 0, nullptr, 0, 1.0)) != cudaSuccess || (e = sweep1(liy, P(5), P(6))) != cudaSuccess ||
        (e = lin1(P(7), ny, P(6), -1.0, nullptr, 0, 1.0)) != cudaSuccess ||
        (e = lin1(P(8), ny, P(6), 2.0 * bg - 1.0, nullptr, 0, 1.0 - bg)) != cudaSuccess ||
        (e = lin1(P(9), ny, P(6), 1.0 - bg, nullptr, 0, 0.0)) != cudaSuccess ||
        (e = sweep1(loy, P(6), P(10))) != cudaSuccess || (e = sweep1(loy, P(7), P(11))) != cudaSuccess ||
        (e = sweep1(loy, P(8), P(12))) != cudaSuccess || (e = sweep1(loy, P(9), P(13))) != cudaSuccess)
        return e;
    // row weights of the four products: 14 = psi2 + H_oy p1 - a2 (with psi1), 15 = -H_oy a2 (with
    // phi_ix), 13 = H_oy p0 - phi_iy (with phi_ox), 10 = -psi2 (with 1)
    if ((e = molt::lincomb<double>(P(14), ny, P(10), 1.0, P(12), 1.0, P(7), -1.0, nullptr, 0, 0.0, st, launches)) !=
            cudaSuccess ||
        (e = lin1(P(15), ny, P(11), -1.0, nullptr, 0, 0.0)) != cudaSuccess ||
        (e = lin1(P(13), ny, P(13), 1.0, P(6), -1.0, 0.0)) != cudaSuccess ||
        (e = lin1(P(10), ny, P(10), -1.0, nullptr, 0, 0.0)) != cudaSuccess)
        return e;
    *out = Separable{{P(14), P(15), P(13), P(10)}, {P(3), P(1), P(2), P(0)}, 4};
    return cudaSuccess;
}

namespace {

using molt::StageParams;
using molt::grid_h;
using molt::stage_params;

}  // namespace

namespace molt {

static bool next_event(Prof* p, int* idx) {
    if (p->used == p->pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return false;
        p->pool.push_back(e);
    }
    *idx = static_cast<int>(p->used++);
    return true;
}

bool Prof::begin(int slot, cudaStream_t st) {
    int a, b;
    if (!next_event(this, &a) || !next_event(this, &b)) return false;
    cudaEventRecord(pool[a], st);
    marks.push_back({slot, a, b});
    return true;
}

void Prof::end(cudaStream_t st) {
    if (!marks.empty()) cudaEventRecord(pool[marks.back().b], st);
}

cudaError_t Prof::collect(double* ms, long long* count) {
    for (int i = 0; i < kProfSlots; ++i) {
        ms[i] = 0.0;
        count[i] = 0;
    }
    for (const Mark& m : marks) {
        cudaError_t e = cudaEventSynchronize(pool[m.b]);
        if (e != cudaSuccess) return e;
        float t = 0.f;
        e = cudaEventElapsedTime(&t, pool[m.a], pool[m.b]);
        if (e != cudaSuccess) return e;
        if (m.slot >= 0 && m.slot < kProfSlots) {
            ms[m.slot] += t;
            count[m.slot] += 1;
        }
    }
    marks.clear();
    used = 0;
    return cudaSuccess;
}

void Prof::release() {
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
    pool.clear();
    marks.clear();
    used = 0;
}

}  // namespace molt

// Precision-independent part of the solver handle.
struct molt_solver {
    molt_grid g;
    molt_params p;
    int bc;
    int device = 0;
    std::string err;
    long long launches = 0;
    molt::Prof prof;
    int exec_mode = MOLT_EXEC_GRAPH;
    long long graph_fallbacks = 0;
    // history
    bool have_prev = false;
    double dt_prev = 0.0;
    bool have_prev2 = false;     // a second earlier level (BDF3)
    double dt_prev2 = 0.0;
    bool have_sdc = false;
    bool have_adapt_prev = false;  // BE-BDF2 estimate: state before the last accepted adaptive step
    double dt_adapt_prev = 0.0;    // and that step's size
    bool vch_have_prev = false;    // vector CH BDF2: previous level held
    double vch_dt_prev = 0.0;
    bool vch_adapt_have_prev = false;   // vector BE-BDF2 estimate: state before the last accepted step
    double vch_adapt_dt_prev = 0.0;     // and that step's size
    virtual ~molt_solver() { prof.release(); }
    virtual molt_status step(void* u, double dt, int scheme, cudaStream_t st, molt_step_info* info) = 0;
    virtual molt_status run_host(void* u_host, double dt, int scheme, int nsteps, cudaStream_t st,
                                 molt_step_info* info) = 0;
    virtual molt_status reduce(const void* u, int which, double* out, cudaStream_t st) = 0;
    virtual molt_status adaptive(void* u, double dt, const molt_adaptive& a, cudaStream_t st,
                                 molt_adaptive_info* info) = 0;
    virtual molt_status vch_step(void* u1, void* u2, double dt, int scheme, cudaStream_t st,
                                 molt_step_info* info) = 0;
    virtual molt_status vch_adaptive(void* u1, void* u2, double dt, const molt_adaptive& a, cudaStream_t st,
                                     molt_adaptive_info* info) = 0;
    virtual molt_status apply(int axis, double c, const void* in, void* out, cudaStream_t st) = 0;
    virtual molt_status apply_tc(double c, const void* in, void* out, cudaStream_t st) = 0;
    virtual molt_status autotune(cudaStream_t st, molt_tuning* out, int capacity, int* nout) = 0;
    virtual molt_status init() = 0;
    virtual void drop_graphs() = 0;
};

namespace {

// Step-size control of Algorithm 1 (Sec. 5), with r = eta / lte_tol and q = N_it / N_maxit.
// A step is accepted when r <= 1 and q < 1.  The next size is dt times a factor: the LTE proposal
// theta / sqrt(r), capped at gamma while q < 0.7 and at 1 while q < 1 for an accepted step; a
// rejected step retries with dt / gamma when the LTE was met (so the iteration hit its cap) or
// r > 2, and with the LTE proposal for 1 < r <= 2.  The result is clipped to [dt_min, dt_max].
// Returns whether the step is accepted.
bool step_size_rule(double eta, int n_it, double dt, const molt_adaptive& a, double* next, int max_iter) {
    const double r = eta / a.lte_tol, q = static_cast<double>(n_it) / max_iter;
    const double proposal = eta == 0.0 ? INFINITY : a.theta / std::sqrt(r);
    const bool accept = r <= 1.0 && q < 1.0;
    double factor;
    if (accept) factor = std::min(proposal, q < 0.7 ? a.gamma : 1.0);
    else factor = (r <= 1.0 || r > 2.0) ? 1.0 / a.gamma : proposal;
    *next = std::min(std::max(dt * factor, a.dt_min), a.dt_max);
    return accept;
}

template <typename T>
struct Solver final : molt_solver {
    // device fields (nx*ny elements each)
    T *w = nullptr, *wn = nullptr, *wprev = nullptr, *r = nullptr, *Y = nullptr;
    T *f1 = nullptr, *f2 = nullptr, *f3 = nullptr, *f4 = nullptr, *f5 = nullptr, *f6 = nullptr;
    T *k0 = nullptr, *k1 = nullptr, *ubuf = nullptr;
    T *wprev2 = nullptr;                      // stored variable two levels back (BDF3)
    T *sdc_w0 = nullptr, *sdc_F0 = nullptr;   // SDC2: level-[0] state and its F
    // vector CH (allocated on first use): second component's state, Y, start of step, previous
    // level and right side, the pass outputs the second component keeps until its last pass, and
    // the first component's previous level
    T *vw2 = nullptr, *vY2 = nullptr, *vn2 = nullptr, *vp2 = nullptr, *vr2 = nullptr;
    T *vg4 = nullptr, *vg5 = nullptr, *vg6 = nullptr, *vp1 = nullptr;
    molt::ColScratch<T> cs{};
    unsigned long long* red = nullptr;       // device [2]
    unsigned long long* red_host = nullptr;  // pinned [2]
    unsigned* wait_status = nullptr;         // device [1]: set by kernels whose bounded waits ran out
    unsigned* wait_status_host = nullptr;    // pinned [1]
    double* dprof = nullptr;                 // device [kProfiles][max(nx, ny)]: Dirichlet offset profiles
    double* partials = nullptr;              // device [reduce_blocks]
    double* result = nullptr;                // device [1]
    double* result_host = nullptr;           // pinned [1]
    std::vector<void*> allocs;

    size_t count() const { return static_cast<size_t>(g.nx) * g.ny; }
    bool fp32() const { return sizeof(T) == 4; }
    T shift() const { return T(1); }     // stored w = v - 1 (see the file comment)

    ~Solver() override {
        drop_graphs();
        if (cap_stream) cudaStreamDestroy(cap_stream);
        if (ls_host) cudaFreeHost(ls_host);
        for (void* a : allocs) cudaFree(a);
        if (red_host) cudaFreeHost(red_host);
        if (result_host) cudaFreeHost(result_host);
        if (wait_status_host) cudaFreeHost(wait_status_host);
    }

    molt_status fail(molt_status s, const std::string& m) {
        err = m;
        return s;
    }
    // A column kernel's copy did not complete within its time limit; its outputs are invalid.
    // The status stays set, so every later step of this solver reports the same error.
    molt_status wait_timeout() {
        err = "a device-side wait for a tile copy ran out of time; results of this step are invalid";
        return MOLT_ERR_CUDA;
    }
    molt_status cuda_fail(cudaError_t e, const char* where) {
        err = std::string(where) + ": " + cudaGetErrorString(e);
        return MOLT_ERR_CUDA;
    }

    template <typename U>
    bool alloc(U** p, size_t n) {
        void* q = nullptr;
        if (cudaMalloc(&q, n * sizeof(U)) != cudaSuccess) return false;
        allocs.push_back(q);
        *p = static_cast<U*>(q);
        return true;
    }

    molt_status init() override {
        const size_t n = count();
        T** fields[] = {&w, &wn, &wprev, &wprev2, &r, &Y, &f1, &f2, &f3, &f4, &f5, &f6, &k0, &k1, &sdc_w0, &sdc_F0};
        for (T** f : fields)
            if (!alloc(f, n)) return fail(MOLT_ERR_OOM, "device workspace allocation failed");
        const int nlines = g.nx;
        const int tiles = (g.ny + 127) / 128;
        cs.tiles = tiles;
        cs.capacity_lines = nlines;
        cs.capacity_fields = 2;
        const size_t sc = static_cast<size_t>(2) * tiles * nlines;
        if (!alloc(&cs.aggL, sc) || !alloc(&cs.aggR, sc) || !alloc(&cs.carL, sc) || !alloc(&cs.carR, sc) ||
            !alloc(&red, 2) || !alloc(&partials, static_cast<size_t>(molt::reduce_blocks())) || !alloc(&result, 1) ||
            !alloc(&dprof, static_cast<size_t>(kProfiles) * std::max(g.nx, g.ny)))
            return fail(MOLT_ERR_OOM, "device scratch allocation failed");
        if (!alloc(&ls, 1)) return fail(MOLT_ERR_OOM, "device loop state allocation failed");
        if (!alloc(&wait_status, 1)) return fail(MOLT_ERR_OOM, "device status allocation failed");
        if (cudaMemset(wait_status, 0, sizeof(unsigned)) != cudaSuccess)
            return fail(MOLT_ERR_CUDA, "device status initialisation failed");
        cs.status = wait_status;
        if (cudaMallocHost(&red_host, 2 * sizeof(unsigned long long)) != cudaSuccess ||
            cudaMallocHost(&result_host, sizeof(double)) != cudaSuccess ||
            cudaMallocHost(&ls_host, sizeof(molt::LoopState)) != cudaSuccess ||
            cudaMallocHost(&wait_status_host, sizeof(unsigned)) != cudaSuccess)
            return fail(MOLT_ERR_OOM, "pinned host allocation failed");
        *wait_status_host = 0;
        return MOLT_OK;
    }

    bool line_params(double c, int axis, molt::LineParams<T>* out) {
        molt::LineParams<double> lp;
        const char* e = nullptr;
        const int n = axis == 0 ? g.nx : g.ny;
        const double L = axis == 0 ? g.Lx : g.Ly;
        if (!molt::build_line_params(c, grid_h(n, L, bc), n, p.quad_order, bc, &lp, &e)) {
            err = e ? e : "line parameters";
            return false;
        }
        *out = molt::cast_line_params<T>(lp);
        return true;
    }

    // Launch choice of each (pass kind, axis), set by the autotuner (molt_autotune); 0 = default.
    int tune[10][2] = {};

    cudaError_t sweep(int axis, const molt::LineParams<T>& lp, int kind, const molt::OpArgs<T>& a,
                      cudaStream_t st) {
        if (a.variant == 0 && kind >= 0 && kind < 10 && tune[kind][axis] != 0 &&
            tune[kind][axis] != molt::LAUNCH_ROWS_TENSOR_CORE) {
            molt::OpArgs<T> b = a;
            b.variant = tune[kind][axis];
            return molt::sweep<T>(axis, lp, kind, b, g.nx, g.ny, &cs, red, st, &launches, &prof);
        }
        return molt::sweep<T>(axis, lp, kind, a, g.nx, g.ny, &cs, red, st, &launches, &prof);
    }

    // One H_c sweep; c (when given) lets the tuned tensor-core row sweep build its operands.
    cudaError_t copy_sweep(int axis, const molt::LineParams<T>& lp, const T* in, T* out, cudaStream_t st,
                           double c = 0.0) {
        if (axis == 0 && c > 0.0 && tune[molt::OP_COPY][0] == molt::LAUNCH_ROWS_TENSOR_CORE && in != out) {
            const cudaError_t e = tc_sweep(c, in, out, st);
            if (e != cudaErrorNotReady) return e;   // not ready during stream capture: the scan kernel
        }
        molt::OpArgs<T> a;
        a.in0 = in;
        a.out0 = out;
        return sweep(axis, lp, molt::OP_COPY, a, st);
    }

    // Tensor-core row sweep with operands cached per c (four slots); the operands are built (host
    // FP64, one synchronizing upload) outside stream capture only.
    struct TcSlot {
        double c = 0.0;
        void* work = nullptr;
    };
    TcSlot tc_slots[4];
    int tc_next = 0;
    cudaError_t tc_sweep(double c, const T* in, T* out, cudaStream_t st) {
        if constexpr (!std::is_same<T, float>::value) {
            return cudaErrorInvalidValue;
        } else {
            const double h = grid_h(g.nx, g.Lx, bc);
            molt::LineParams<double> lpd;
            const char* err = nullptr;
            if (!molt::build_line_params(c, h, g.nx, p.quad_order, bc, &lpd, &err)) return cudaErrorInvalidValue;
            TcSlot* slot = nullptr;
            for (TcSlot& t : tc_slots)
                if (t.work && t.c == c) slot = &t;
            if (!slot) {
                cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
                if (cudaStreamIsCapturing(st, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) {
                    cudaGetLastError();
                    return cudaErrorNotReady;
                }
                slot = &tc_slots[tc_next];
                tc_next = (tc_next + 1) % 4;
                if (!slot->work) {
                    if (cudaMalloc(&slot->work, molt::rows_tc_workspace_bytes()) != cudaSuccess)
                        return cudaErrorMemoryAllocation;
                    allocs.push_back(slot->work);
                }
                slot->c = c;
                const cudaError_t e = molt::rows_tc_prepare(lpd, slot->work, st);
                if (e != cudaSuccess) {
                    slot->c = 0.0;
                    return e;
                }
            }
            launches += 1;
            return molt::rows_tc(lpd, slot->work, in, out, g.ny, wait_status, st);
        }
    }

    cudaError_t lin(T* out, const T* x0, double c0, const T* x1 = nullptr, double c1 = 0, const T* x2 = nullptr,
                    double c2 = 0, const T* x3 = nullptr, double c3 = 0, double c4 = 0, cudaStream_t st = nullptr) {
        return molt::lincomb<T>(out, static_cast<long long>(count()), x0, c0, x1, c1, x2, c2, x3, c3, c4, st,
                                &launches);
    }

    // out = M_c^{-1} in = H_x H_y in (2D) or H_x in (1D); uses f1 as scratch in 2D.
    cudaError_t mm_inv(double c, const T* in, T* out, cudaStream_t st) {
        molt::LineParams<T> lx, ly;
        if (!line_params(c, 0, &lx)) return cudaErrorInvalidValue;
        if (g.dim == 1) return copy_sweep(0, lx, in, out, st, c);
        if (!line_params(c, 1, &ly)) return cudaErrorInvalidValue;
        cudaError_t e = copy_sweep(1, ly, in, f1, st);
        if (e != cudaSuccess) return e;
        return copy_sweep(0, lx, f1, out, st, c);
    }

    // out = E_c in with E = M^{-1} - I + D_x D_y, i.e. 2 H_x H_y - H_x - H_y in 2D and H - I in 1D
    // (the operator through which M^{-1} acts on c Lap, Remark Laplacian); scratch f1, f2, f3.
    cudaError_t e_op(double c, const T* in, T* out, cudaStream_t st) {
        molt::LineParams<T> lx, ly;
        if (!line_params(c, 0, &lx)) return cudaErrorInvalidValue;
        cudaError_t e;
        if (g.dim == 1) {
            if ((e = copy_sweep(0, lx, in, f1, st, c)) != cudaSuccess) return e;
            return lin(out, f1, 1.0, in, -1.0, nullptr, 0, nullptr, 0, 0, st);
        }
        if (!line_params(c, 1, &ly)) return cudaErrorInvalidValue;
        if ((e = copy_sweep(1, ly, in, f1, st)) != cudaSuccess) return e;      // H_y
        if ((e = copy_sweep(0, lx, f1, f2, st, c)) != cudaSuccess) return e;   // H_x H_y
        if ((e = copy_sweep(0, lx, in, f3, st, c)) != cudaSuccess) return e;   // H_x
        return lin(out, f2, 2.0, f3, -1.0, f1, -1.0, nullptr, 0, 0, st);
    }

    // out = M_o^{-1} M_i^{-1} F(v) for v stored in w_in, without derivatives (Remark Laplacian /
    // biLaplacian): -(eps^2/(c_i c_o)) E_o E_i v + (1/c_i) M_o^{-1} E_i f(v-1).  E kills constants
    // on periodic / Neumann grids, so E_i v = E_i w there; on Dirichlet grids v = w + 1 is formed
    // first.  f(v-1) = w^3 - w for w = v - 1.  Scratch: f1..f6.
    cudaError_t inverse_of_F(const StageParams& sp, const T* w_in, T* out, cudaStream_t st) {
        cudaError_t e;
        const T* v_in = w_in;
        if (bc == molt::BC_DIRICHLET) {   // Dirichlet E does not kill constants: form v = w + 1
            if ((e = lin(f5, w_in, 1.0, nullptr, 0, nullptr, 0, nullptr, 0, 1.0, st)) != cudaSuccess) return e;
            v_in = f5;
        }
        if ((e = e_op(sp.c_in, v_in, f4, st)) != cudaSuccess) return e;        // E_i v
        if ((e = e_op(sp.c_out, f4, f5, st)) != cudaSuccess) return e;         // E_o E_i v
        const bool shifted = shift() == T(1);
        if ((e = molt::cubic<T>(f6, static_cast<long long>(count()), w_in, shifted ? 0.0 : -3.0,
                                shifted ? -1.0 : 2.0, st, &launches)) != cudaSuccess)
            return e;                                                           // f(v-1)
        if ((e = e_op(sp.c_in, f6, f4, st)) != cudaSuccess) return e;         // E_i f
        if ((e = mm_inv(sp.c_out, f4, f6, st)) != cudaSuccess) return e;      // M_o^{-1} E_i f
        return lin(out, f5, -(p.eps * p.eps) / (sp.c_in * sp.c_out), f6, 1.0 / sp.c_in, nullptr, 0, nullptr, 0, 0,
                   st);
    }

    // Dirichlet grids: the fixed field C the constant part of v adds to each stage's Y (see the file
    // comment and molt::dirichlet_offset), added per point in FP64.
    static constexpr int kProfiles = molt::kOffsetProfiles;
    cudaError_t add_dirichlet_offset(const StageParams& sp, T* y, cudaStream_t st) {
        molt::LineParams<double> lp[4];
        const double cs[4] = {sp.c_in, sp.c_out, sp.c_in, sp.c_out};
        for (int k = 0; k < (g.dim == 2 ? 4 : 2); ++k) {
            const int axis = k / 2, n = axis == 0 ? g.nx : g.ny;
            const char* e = nullptr;
            if (!molt::build_line_params(cs[k], grid_h(n, axis == 0 ? g.Lx : g.Ly, bc), n, p.quad_order, bc, &lp[k], &e))
                return cudaErrorInvalidValue;
        }
        molt::Separable sep;
        const cudaError_t e = molt::dirichlet_offset(lp, g.dim, sp.beta * (sp.lam - 2.0), dprof, std::max(g.nx, g.ny),
                                                     &sep, st, &launches);
        if (e != cudaSuccess) return e;
        return molt::add_separable<T>(y, g.nx, g.dim == 2 ? g.ny : 1, sep, st, &launches);
    }

    // Everything one fixed-point iteration of a stage launches (line parameters by value).
    struct Passes {
        molt::LineParams<T> lix, lox, liy, loy;
        T g2, g1, beta, s;
        bool two_d;
        bool vch = false;   // vector CH iteration (both components)
        T vs = 0;           // vector CH: (c1 + c2)/tau
    };

    bool make_passes(const StageParams& sp, Passes* ps) {
        ps->two_d = g.dim == 2;
        if (!line_params(sp.c_in, 0, &ps->lix) || !line_params(sp.c_out, 0, &ps->lox)) return false;
        if (ps->two_d && (!line_params(sp.c_in, 1, &ps->liy) || !line_params(sp.c_out, 1, &ps->loy))) return false;
        ps->s = shift();
        ps->g2 = ps->s == T(1) ? T(0) : T(-3);
        ps->g1 = ps->s == T(1) ? static_cast<T>(sp.lam - 3.0) : static_cast<T>(sp.lam);
        ps->beta = static_cast<T>(sp.beta);
        return true;
    }

    // Vector CH stage (Sec. 5.2): the factorization of Eq. CH_vector_fixed1 for tau >= eps^2/81
    // (c = 9 tau +- sqrt(81 tau^2 - eps^2 tau)), else the completed square of Eq. CH_vector_fixed2
    // (c1 = c2 = sqrt(eps^2 tau)); s = (c1 + c2)/tau.
    bool make_vch_passes(double tau, Passes* ps, double* c_in, double* c_out) {
        const double e2 = p.eps * p.eps;
        double c1, c2;
        if (81.0 * tau >= e2) {
            const double disc = std::sqrt(81.0 * tau * tau - e2 * tau);
            c1 = 9.0 * tau + disc;
            c2 = 9.0 * tau - disc;
        } else {
            c1 = c2 = std::sqrt(e2 * tau);
        }
        *c_in = std::max(c1, c2);
        *c_out = std::min(c1, c2);
        ps->two_d = g.dim == 2;
        if (!line_params(*c_in, 0, &ps->lix) || !line_params(*c_out, 0, &ps->lox)) return false;
        if (ps->two_d && (!line_params(*c_in, 1, &ps->liy) || !line_params(*c_out, 1, &ps->loy))) return false;
        ps->s = shift();
        ps->g2 = ps->g1 = T(0);
        ps->beta = static_cast<T>(tau / *c_in);
        ps->vch = true;
        ps->vs = static_cast<T>((c1 + c2) / tau);
        return true;
    }

    // One vector CH iteration.  Both components' lagged terms come from the previous iterate, so
    // every pass that reads both state fields runs before either is overwritten: passes 1-3 of
    // each component, then pass 4 of each (2D); pass a of each, then pass b of each (1D).
    cudaError_t launch_vch_iteration(const Passes& ps, cudaStream_t st) {
        cudaError_t e;
        T* V[2] = {w, vw2};
        const T* Yc[2] = {Y, vY2};
        if (ps.two_d) {
            T* U[2] = {f4, vg4};
            T* Q1[2] = {f5, vg5};
            T* Q2[2] = {f6, vg6};
            for (int c = 0; c < 2; ++c) {
                molt::OpArgs<T> a1;
                a1.in0 = w; a1.in1 = vw2; a1.out0 = f1; a1.out1 = f2; a1.vs = ps.vs; a1.comp = c;
                if ((e = sweep(1, ps.liy, molt::OP_V1, a1, st)) != cudaSuccess) return e;
                molt::OpArgs<T> a2;
                a2.in0 = w; a2.in1 = vw2; a2.in2 = f1; a2.in3 = f2; a2.out0 = f3; a2.out1 = U[c];
                a2.vs = ps.vs; a2.beta = ps.beta; a2.comp = c;
                if ((e = sweep(0, ps.lix, molt::OP_V2, a2, st)) != cudaSuccess) return e;
                molt::OpArgs<T> a3;
                a3.in0 = f3; a3.in1 = U[c]; a3.out0 = Q1[c]; a3.out1 = Q2[c];
                if ((e = sweep(1, ps.loy, molt::OP_P3, a3, st)) != cudaSuccess) return e;
            }
            for (int c = 0; c < 2; ++c) {
                molt::OpArgs<T> a4;
                a4.in0 = Q1[c]; a4.in1 = Q2[c]; a4.in2 = U[c]; a4.in3 = Yc[c]; a4.out0 = V[c]; a4.shift = ps.s;
                if ((e = sweep(0, ps.lox, molt::OP_P4, a4, st)) != cudaSuccess) return e;
                if ((e = impose_walls(V[c], st, 0.0)) != cudaSuccess) return e;
            }
            return cudaSuccess;
        }
        T* E[2] = {f1, f2};
        for (int c = 0; c < 2; ++c) {
            molt::OpArgs<T> aa;
            aa.in0 = w; aa.in1 = vw2; aa.out0 = E[c]; aa.vs = ps.vs; aa.beta = ps.beta; aa.comp = c;
            if ((e = sweep(0, ps.lix, molt::OP_V1A, aa, st)) != cudaSuccess) return e;
        }
        for (int c = 0; c < 2; ++c) {
            molt::OpArgs<T> ab;
            ab.in0 = E[c]; ab.in1 = Yc[c]; ab.out0 = V[c]; ab.shift = ps.s;
            if ((e = sweep(0, ps.lox, molt::OP_1B, ab, st)) != cudaSuccess) return e;
            if ((e = impose_walls(V[c], st, 0.0)) != cudaSuccess) return e;
        }
        return cudaSuccess;
    }

    // Dirichlet grids: every line inverse holds v = 0 on the walls exactly, so every iterate does; the
    // stored wall value w = v - 1 = -1 is set after each iteration instead of carrying the FP32
    // rounding of the sum of O(1) terms that reproduces it (the vector model stores v - z3 = 0).
    cudaError_t impose_walls(T* field, cudaStream_t st, double value = -1.0) {
        if (bc != molt::BC_DIRICHLET) return cudaSuccess;
        return molt::set_walls<T>(field, g.nx, g.dim == 2 ? g.ny : 1, value, st, &launches);
    }

    // One iteration: 2D passes 1-4 (column, row, column, row) or the two 1D row passes.  The
    // last pass accumulates the residual into `red`.
    cudaError_t launch_iteration(const Passes& ps, cudaStream_t st) {
        if (ps.vch) return launch_vch_iteration(ps, st);
        cudaError_t e;
        if (ps.two_d) {
            // Block orders alternate so that each pass starts at the end of the field the pass
            // before it finished on (still in L2): pass 4 ends at the last row, pass 1 aggregates
            // from the last tile row up and finishes from the first down, pass 2 runs from the
            // last line up, pass 3 aggregates from the first tile row down and finishes from the
            // last up, and pass 4 starts again at the first line.
            molt::OpArgs<T> a1;
            a1.in0 = w; a1.out0 = f1; a1.out1 = f2; a1.g2 = ps.g2; a1.g1 = ps.g1; a1.order = 1;
            if ((e = sweep(1, ps.liy, molt::OP_P1, a1, st)) != cudaSuccess) return e;
            molt::OpArgs<T> a2;
            a2.in0 = w; a2.in1 = f1; a2.in2 = f2; a2.out0 = f3; a2.out1 = f4;
            a2.g2 = ps.g2; a2.g1 = ps.g1; a2.beta = ps.beta; a2.order = 1;
            if ((e = sweep(0, ps.lix, molt::OP_P2, a2, st)) != cudaSuccess) return e;
            molt::OpArgs<T> a3;
            a3.in0 = f3; a3.in1 = f4; a3.out0 = f5; a3.out1 = f6; a3.order = 2;
            if ((e = sweep(1, ps.loy, molt::OP_P3, a3, st)) != cudaSuccess) return e;
            molt::OpArgs<T> a4;
            a4.in0 = f5; a4.in1 = f6; a4.in2 = f4; a4.in3 = Y; a4.out0 = w; a4.shift = ps.s;
            if ((e = sweep(0, ps.lox, molt::OP_P4, a4, st)) != cudaSuccess) return e;
            return impose_walls(w, st);
        }
        molt::OpArgs<T> aa;
        aa.in0 = w; aa.out0 = f1; aa.g2 = ps.g2; aa.g1 = ps.g1; aa.beta = ps.beta;
        if ((e = sweep(0, ps.lix, molt::OP_1A, aa, st)) != cudaSuccess) return e;
        molt::OpArgs<T> ab;
        ab.in0 = f1; ab.in1 = Y; ab.out0 = w; ab.shift = ps.s;
        if ((e = sweep(0, ps.lox, molt::OP_1B, ab, st)) != cudaSuccess) return e;
        return impose_walls(w, st);
    }

    // Executable graphs of the stage loop, one per stage coefficient tau: a conditional WHILE
    // node whose body is one iteration followed by the device-side stopping check.
    struct LoopGraph {
        bool valid = false;
        bool vch = false;
        double tau = 0.0;
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        long long kernels_per_iter = 0;
    };
    static constexpr int kGraphSlots = 4;
    LoopGraph graphs[kGraphSlots];
    int next_graph = 0;
    cudaStream_t cap_stream = nullptr;
    molt::LoopState* ls = nullptr;
    molt::LoopState* ls_host = nullptr;

    void drop_graphs() override {
        for (LoopGraph& lg : graphs) {
            if (lg.exec) cudaGraphExecDestroy(lg.exec);
            if (lg.graph) cudaGraphDestroy(lg.graph);
            lg = LoopGraph();
        }
    }

    LoopGraph* loop_graph(double tau, const Passes& ps) {
        for (LoopGraph& lg : graphs)
            if (lg.valid && lg.tau == tau && lg.vch == ps.vch) return &lg;
        LoopGraph& lg = graphs[next_graph];
        next_graph = (next_graph + 1) % kGraphSlots;
        if (lg.exec) cudaGraphExecDestroy(lg.exec);
        if (lg.graph) cudaGraphDestroy(lg.graph);
        lg = LoopGraph();
        if (!cap_stream && cudaStreamCreateWithFlags(&cap_stream, cudaStreamNonBlocking) != cudaSuccess) return nullptr;
        cudaGraph_t graph = nullptr;
        if (cudaGraphCreate(&graph, 0) != cudaSuccess) return nullptr;
        cudaGraphConditionalHandle h;
        cudaGraphNodeParams np = {};
        np.type = cudaGraphNodeTypeConditional;
        cudaGraphNode_t node;
        bool ok = cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault) == cudaSuccess;
        if (ok) {
            np.conditional.handle = h;
            np.conditional.type = cudaGraphCondTypeWhile;
            np.conditional.size = 1;
            ok = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &np) == cudaSuccess;
        }
        const long long before = launches;
        if (ok) {
            cudaGraph_t body = np.conditional.phGraph_out[0];
            ok = cudaStreamBeginCaptureToGraph(cap_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) ==
                 cudaSuccess;
            if (ok) {
                const bool launched =
                    launch_iteration(ps, cap_stream) == cudaSuccess &&
                    molt::loop_check(h, ls, red, p.tol, p.max_iter, fp32() ? 1 : 0, cap_stream) == cudaSuccess;
                cudaGraph_t captured = nullptr;
                ok = cudaStreamEndCapture(cap_stream, &captured) == cudaSuccess && launched;
            }
        }
        lg.kernels_per_iter = launches - before + 1;
        launches = before;
        cudaGraphExec_t exec = nullptr;
        if (ok) ok = cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            if (exec) cudaGraphExecDestroy(exec);
            cudaGraphDestroy(graph);
            return nullptr;
        }
        lg.valid = true;
        lg.vch = ps.vch;
        lg.tau = tau;
        lg.graph = graph;
        lg.exec = exec;
        return &lg;
    }

    // Solve v - tau F(v) = r for w (in: first guess, out: last iterate), r in stored form.
    // With y_given, the field Y already holds M_o^{-1} M_i^{-1} r and rhs is not read.
    // With `given`, its passes are run (the vector CH stage) and Y must be given.
    molt_status stage(double tau, const T* rhs, cudaStream_t st, int* iters, double* res_out, double* tol_out,
                      bool y_given = false, const Passes* given = nullptr) {
        const StageParams sp = stage_params(tau, p.eps);
        Passes ps;
        if (given) ps = *given;
        else if (!make_passes(sp, &ps)) return MOLT_ERR_ARG;
        cudaError_t e = cudaSuccess;
        if (!y_given) {
            // Y = M_o^{-1} M_i^{-1} r
            if ((e = mm_inv(sp.c_in, rhs, f2, st)) != cudaSuccess) return cuda_fail(e, "rhs inverse");
            if ((e = mm_inv(sp.c_out, f2, Y, st)) != cudaSuccess) return cuda_fail(e, "rhs inverse");
        }
        if (!given && bc == molt::BC_DIRICHLET && (e = add_dirichlet_offset(sp, Y, st)) != cudaSuccess)
            return cuda_fail(e, "Dirichlet offset");
        if (exec_mode == MOLT_EXEC_GRAPH && !prof.on) {
            LoopGraph* lg = loop_graph(tau, ps);
            if (lg) {
                // the whole loop on the device; one read-back of the loop state per stage
                if ((e = molt::loop_init(ls, red, st)) != cudaSuccess) return cuda_fail(e, "loop init");
                if ((e = cudaGraphLaunch(lg->exec, st)) != cudaSuccess) return cuda_fail(e, "graph launch");
                if ((e = cudaMemcpyAsync(ls_host, ls, sizeof(molt::LoopState), cudaMemcpyDeviceToHost, st)) !=
                    cudaSuccess)
                    return cuda_fail(e, "loop state copy");
                if ((e = cudaMemcpyAsync(wait_status_host, wait_status, sizeof(unsigned), cudaMemcpyDeviceToHost,
                                         st)) != cudaSuccess)
                    return cuda_fail(e, "status copy");
                if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "stream sync");
                if (*wait_status_host) return wait_timeout();
                launches += 1 + static_cast<long long>(ls_host->k) * lg->kernels_per_iter;
                *iters = ls_host->k;
                *res_out = ls_host->res;
                *tol_out = ls_host->tol_used;
                return ls_host->converged ? MOLT_OK : MOLT_ERR_NOT_CONVERGED;
            }
            graph_fallbacks += 1;     // graph construction failed: run the host-driven loop
        }
        double res = INFINITY, tol_used = p.tol, best = INFINITY;
        int k = 0, stall = 0;
        bool converged = false;
        for (k = 1; k <= p.max_iter; ++k) {
            if ((e = cudaMemsetAsync(red, 0, 2 * sizeof(unsigned long long), st)) != cudaSuccess)
                return cuda_fail(e, "memset");
            if ((e = launch_iteration(ps, st)) != cudaSuccess) return cuda_fail(e, "iteration");
            if ((e = cudaMemcpyAsync(red_host, red, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st)) !=
                cudaSuccess)
                return cuda_fail(e, "residual copy");
            if ((e = cudaMemcpyAsync(wait_status_host, wait_status, sizeof(unsigned), cudaMemcpyDeviceToHost, st)) !=
                cudaSuccess)
                return cuda_fail(e, "status copy");
            if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "stream sync");
            if (*wait_status_host) return wait_timeout();
            double dmax, wmax;
            std::memcpy(&dmax, &red_host[0], sizeof(double));
            std::memcpy(&wmax, &red_host[1], sizeof(double));
            res = dmax;
            if (!std::isfinite(res)) break;
            // FP32 fields cannot resolve changes below a few units in the last place of the
            // stored variable: the tolerance is floored at 2 ulp of max|w| (see the stall rule below).
            const double ulp = std::ldexp(1.0, -24) * wmax;
            tol_used = fp32() ? std::max(p.tol, 2.0 * ulp) : p.tol;
            if (res < tol_used) {
                converged = true;
                break;
            }
            // A steadily (even slowly) contracting iteration keeps lowering its residual; one
            // that has not set a new minimum for 6 iterations while below 64 ulp is at the FP32
            // noise floor.
            if (res < best) {
                best = res;
                stall = 0;
            } else if (fp32() && res < 64.0 * ulp && ++stall >= 6) {
                converged = true;
                tol_used = res;
                break;
            }
        }
        *iters = converged ? k : std::min(k, p.max_iter);
        *res_out = res;
        *tol_out = tol_used;
        return converged ? MOLT_OK : MOLT_ERR_NOT_CONVERGED;
    }

    void record(molt_step_info* info, int stage_idx, int it, double res, double tol_used) {
        if (!info) return;
        if (stage_idx < 4) info->iters[stage_idx] = it;
        info->stages = stage_idx + 1;
        info->total_iters += it;
        info->residual = std::max(info->residual, res);
        info->tol_used = tol_used;
    }

    molt_status sdirk(double dt, const double A[3][3], int s_count, cudaStream_t st, molt_step_info* info,
                      int stage0) {
        // stage-value form: V_i - eta dt F(V_i) = w^n + dt sum_{l<i} a_il K_l, K_l = (V_l - R_l)/(eta dt)
        const double eta = A[0][0];
        T* K[2] = {k0, k1};
        molt_status worst = MOLT_OK;
        cudaError_t e;
        for (int i = 0; i < s_count; ++i) {
            if (i == 0) e = lin(r, wn, 1.0, nullptr, 0, nullptr, 0, nullptr, 0, 0, st);
            else if (i == 1) e = lin(r, wn, 1.0, K[0], dt * A[1][0], nullptr, 0, nullptr, 0, 0, st);
            else e = lin(r, wn, 1.0, K[0], dt * A[2][0], K[1], dt * A[2][1], nullptr, 0, 0, st);
            if (e != cudaSuccess) return cuda_fail(e, "stage rhs");
            int it;
            double res, tu;
            molt_status ms = stage(eta * dt, r, st, &it, &res, &tu);
            if (ms != MOLT_OK && ms != MOLT_ERR_NOT_CONVERGED) return ms;
            if (ms != MOLT_OK) worst = ms;
            record(info, stage0 + i, it, res, tu);
            if (i + 1 < s_count) {
                if ((e = lin(K[i], w, 1.0 / (eta * dt), r, -1.0 / (eta * dt), nullptr, 0, nullptr, 0, 0, st)) !=
                    cudaSuccess)
                    return cuda_fail(e, "stage slope");
            }
        }
        return worst;
    }

    // SDC2 (Sec. 4.3, Eq. IDC_BE_j with the trapezoid rule, Eq. SDC_fixed): the level-[0] BE
    // trajectory and the level-[1] correction advance together.  Level [1] solves
    //   v1_{n+1} - dt F(v1_{n+1}) = v1_n - (dt/2)(F0_{n+1} - F0_n),
    // with F0_{n+1} = (v0_{n+1} - v0_n)/dt from the BE identity and, at a (re)start, F0_n taken
    // inside the inverse (inverse_of_F).  Level [1] starts from the level-[0] value.
    molt_status sdc2(double dt, cudaStream_t st, molt_step_info* info) {
        const bool start = !have_sdc || dt_prev != dt;
        const StageParams sp = stage_params(dt, p.eps);
        const T* v0n = start ? wn : sdc_w0;
        cudaError_t e;
        if ((e = lin(w, v0n, 1.0, nullptr, 0, nullptr, 0, nullptr, 0, 0, st)) != cudaSuccess)
            return cuda_fail(e, "sdc guess");
        int it;
        double res, tu;
        molt_status worst = MOLT_OK;
        molt_status ms = stage(dt, v0n, st, &it, &res, &tu);                  // level [0]: BE
        if (ms != MOLT_OK && ms != MOLT_ERR_NOT_CONVERGED) return ms;
        if (ms != MOLT_OK) worst = ms;
        record(info, 0, it, res, tu);
        if ((e = lin(k0, w, 1.0 / dt, v0n, -1.0 / dt, nullptr, 0, nullptr, 0, 0, st)) != cudaSuccess)
            return cuda_fail(e, "sdc F");                                      // F0_{n+1}
        if ((e = lin(k1, w, 1.0, nullptr, 0, nullptr, 0, nullptr, 0, 0, st)) != cudaSuccess)
            return cuda_fail(e, "sdc state");                                  // v0_{n+1}
        if (start) {
            if ((e = lin(r, wn, 1.0, k0, -0.5 * dt, nullptr, 0, nullptr, 0, 0, st)) != cudaSuccess ||
                (e = mm_inv(sp.c_in, r, f2, st)) != cudaSuccess || (e = mm_inv(sp.c_out, f2, Y, st)) != cudaSuccess ||
                (e = inverse_of_F(sp, v0n, sdc_F0, st)) != cudaSuccess ||
                (e = lin(Y, Y, 1.0, sdc_F0, 0.5 * dt, nullptr, 0, nullptr, 0, 0, st)) != cudaSuccess)
                return cuda_fail(e, "sdc rhs");
        } else {
            if ((e = lin(r, wn, 1.0, k0, -0.5 * dt, sdc_F0, 0.5 * dt, nullptr, 0, 0, st)) != cudaSuccess ||
                (e = mm_inv(sp.c_in, r, f2, st)) != cudaSuccess || (e = mm_inv(sp.c_out, f2, Y, st)) != cudaSuccess)
                return cuda_fail(e, "sdc rhs");
        }
        ms = stage(dt, nullptr, st, &it, &res, &tu, true);                     // level [1]
        if (ms != MOLT_OK && ms != MOLT_ERR_NOT_CONVERGED) return ms;
        if (ms != MOLT_OK) worst = ms;
        record(info, 1, it, res, tu);
        std::swap(sdc_w0, k1);
        std::swap(sdc_F0, k0);
        have_sdc = true;
        return worst;
    }

    molt_status step(void* u_void, double dt, int scheme, cudaStream_t st, molt_step_info* info) override {
        T* u = static_cast<T*>(u_void);
        if (info) std::memset(info, 0, sizeof(*info));
        if (g.dim == 2 && g.nx > molt::max_row_length<T>(2))
            return fail(MOLT_ERR_UNSUPPORTED, "2D steps need x lines within the two-field row kernels' length");
        const double in_shift = 1.0 - static_cast<double>(shift());   // w = u + (1 - s)
        cudaError_t e;
        if ((e = lin(w, u, 1.0, nullptr, 0, nullptr, 0, nullptr, 0, in_shift, st)) != cudaSuccess)
            return cuda_fail(e, "load field");
        if ((e = lin(wn, w, 1.0, nullptr, 0, nullptr, 0, nullptr, 0, 0, st)) != cudaSuccess)
            return cuda_fail(e, "copy field");
        molt_status ms = MOLT_OK;
        int it;
        double res, tu;
        switch (scheme) {
            case MOLT_BE:
                ms = stage(dt, wn, st, &it, &res, &tu);
                record(info, 0, it, res, tu);
                break;
            case MOLT_BDF2:
                if (!have_prev || dt_prev != dt) {
                    ms = stage(dt, wn, st, &it, &res, &tu);          // BE start
                } else {
                    if ((e = lin(r, wn, 4.0 / 3.0, wprev, -1.0 / 3.0, nullptr, 0, nullptr, 0, 0, st)) != cudaSuccess)
                        return cuda_fail(e, "bdf2 rhs");
                    ms = stage(2.0 * dt / 3.0, r, st, &it, &res, &tu);
                }
                record(info, 0, it, res, tu);
                break;
            case MOLT_SDIRK2: {
                const double A[3][3] = {{kEta2, 0, 0}, {1.0 - kEta2, kEta2, 0}, {0, 0, 0}};
                ms = sdirk(dt, A, 2, st, info, 0);
                break;
            }
            case MOLT_SDIRK3: {
                const double eta = alexander_eta();
                const double A[3][3] = {{eta, 0, 0},
                                        {(1.0 - eta) / 2.0, eta, 0},
                                        {-(6 * eta * eta - 16 * eta + 1) / 4.0, (6 * eta * eta - 20 * eta + 5) / 4.0, eta}};
                ms = sdirk(dt, A, 3, st, info, 0);
                break;
            }
            case MOLT_SDC2:
                ms = sdc2(dt, st, info);
                break;
            case MOLT_BDF3:
                if (!have_prev || !have_prev2 || dt_prev != dt || dt_prev2 != dt) {
                    const double A[3][3] = {{kEta2, 0, 0}, {1.0 - kEta2, kEta2, 0}, {0, 0, 0}};
                    ms = sdirk(dt, A, 2, st, info, 0);                 // SDIRK2 start (Sec. 4.4)
                } else {
                    if ((e = lin(r, wn, 18.0 / 11.0, wprev, -9.0 / 11.0, wprev2, 2.0 / 11.0, nullptr, 0, 0, st)) !=
                        cudaSuccess)
                        return cuda_fail(e, "bdf3 rhs");
                    ms = stage(6.0 * dt / 11.0, r, st, &it, &res, &tu);
                    record(info, 0, it, res, tu);
                }
                break;
            default:
                return fail(MOLT_ERR_UNSUPPORTED, "scheme not supported by this build");
        }
        if (scheme != MOLT_SDC2) have_sdc = false;
        if (ms != MOLT_OK && ms != MOLT_ERR_NOT_CONVERGED) return ms;
        // history for BDF2: previous level
        // history: w^{n-2} <- w^{n-1} <- w^n (pointer rotation; wn takes the freed buffer)
        T* freed = wprev2;
        wprev2 = wprev;
        wprev = wn;
        wn = freed;
        have_prev2 = have_prev;
        dt_prev2 = dt_prev;
        have_prev = true;
        dt_prev = dt;
        if ((e = lin(u, w, 1.0, nullptr, 0, nullptr, 0, nullptr, 0, -in_shift, st)) != cudaSuccess)
            return cuda_fail(e, "store field");
        if (info) info->status = ms;
        if (ms == MOLT_ERR_NOT_CONVERGED) err = "a stage reached max_iter before the fixed-point tolerance";
        return ms;
    }

    molt_status run_host(void* u_host, double dt, int scheme, int nsteps, cudaStream_t st,
                         molt_step_info* info) override {
        if (!ubuf && !alloc(&ubuf, count())) return fail(MOLT_ERR_OOM, "device buffer allocation failed");
        const size_t bytes = count() * sizeof(T);
        cudaError_t e;
        if ((e = cudaMemcpyAsync(ubuf, u_host, bytes, cudaMemcpyHostToDevice, st)) != cudaSuccess)
            return cuda_fail(e, "host to device copy");
        molt_status ms = MOLT_OK;
        for (int i = 0; i < nsteps; ++i) {
            ms = step(ubuf, dt, scheme, st, info);
            if (ms != MOLT_OK && ms != MOLT_ERR_NOT_CONVERGED) return ms;
        }
        if ((e = cudaMemcpyAsync(u_host, ubuf, bytes, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
            return cuda_fail(e, "device to host copy");
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "stream sync");
        return ms;
    }

    molt_status reduce(const void* u, int which, double* out, cudaStream_t st) override {
        const double hx = grid_h(g.nx, g.Lx, bc);
        const double hy = g.dim == 2 ? grid_h(g.ny, g.Ly, bc) : 1.0;
        cudaError_t e = molt::energy_mass<T>(static_cast<const T*>(u), g.nx, g.ny, bc, hx, hy, p.eps, which,
                                             partials, result, st, &launches);
        if (e != cudaSuccess) return cuda_fail(e, "reduction");
        if ((e = cudaMemcpyAsync(result_host, result, sizeof(double), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
            return cuda_fail(e, "reduction copy");
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "stream sync");
        *out = *result_host;
        return MOLT_OK;
    }

    // Algorithm 1 (Sec. 5) with the Richardson BE, BE-SDC2 or BE-BDF2 estimate; see
    // include/molt.h for the rules.  The candidate solution of an attempt is built in
    // adapt_half, so u is untouched until a step is accepted.
    T *adapt_full = nullptr, *adapt_half = nullptr, *adapt_prev = nullptr;
    molt_status adaptive(void* u_void, double dt, const molt_adaptive& a, cudaStream_t st,
                         molt_adaptive_info* out) override {
        T* u = static_cast<T*>(u_void);
        const bool want_bdf = a.estimator == MOLT_LTE_BDF2;
        const bool bdf = want_bdf && have_adapt_prev;
        const bool sdc = a.estimator == MOLT_LTE_SDC2 || (want_bdf && !have_adapt_prev);   // BE-BDF2's first step
        if (!adapt_half && !alloc(&adapt_half, count())) return fail(MOLT_ERR_OOM, "adaptive work fields");
        if (!sdc && !adapt_full && !alloc(&adapt_full, count())) return fail(MOLT_ERR_OOM, "adaptive work fields");
        if (want_bdf && !adapt_prev && !alloc(&adapt_prev, count())) return fail(MOLT_ERR_OOM, "adaptive history");
        cudaError_t e;
        int rejections = 0;
        for (;;) {
            molt_step_info i1, i2, i3;
            if ((e = lin(adapt_half, u, 1.0, nullptr, 0, nullptr, 0, nullptr, 0, 0, st)) != cudaSuccess ||
                (!sdc && (e = lin(adapt_full, u, 1.0, nullptr, 0, nullptr, 0, nullptr, 0, 0, st)) != cudaSuccess))
                return cuda_fail(e, "adaptive copy");
            const T* x;   // the two fields whose largest difference gives eta
            const T* y;
            int n_it;
            if (bdf) {
                // One BE step, and one variable-step BDF2 step from (u^{n-1}, u^n) = (adapt_prev, u)
                // with omega = dt / dt_prev:
                //   v - tau F(v) = a_n w^n + a_prev w^{n-1},  tau = dt (1 + omega) / (1 + 2 omega),
                //   a_n = (1 + omega)^2 / (1 + 2 omega),     a_prev = -omega^2 / (1 + 2 omega),
                // the quadratic through the three levels whose slope at t_{n+1} is F(v).
                molt_status s1 = step(adapt_full, dt, MOLT_BE, st, &i1);
                if (s1 != MOLT_OK && s1 != MOLT_ERR_NOT_CONVERGED) return s1;
                const double om = dt / dt_adapt_prev;
                const double tau = dt * (1.0 + om) / (1.0 + 2.0 * om);
                const double an = (1.0 + om) * (1.0 + om) / (1.0 + 2.0 * om), ap = -om * om / (1.0 + 2.0 * om);
                const double in_shift = 1.0 - static_cast<double>(shift());   // w = u + (1 - s)
                if ((e = lin(w, u, 1.0, nullptr, 0, nullptr, 0, nullptr, 0, in_shift, st)) != cudaSuccess ||
                    (e = lin(r, u, an, adapt_prev, ap, nullptr, 0, nullptr, 0, in_shift * (an + ap), st)) !=
                        cudaSuccess)
                    return cuda_fail(e, "bdf2 estimate rhs");
                int it2;
                double res2, tu2;
                molt_status s2 = stage(tau, r, st, &it2, &res2, &tu2);
                if (s2 != MOLT_OK && s2 != MOLT_ERR_NOT_CONVERGED) return s2;
                if ((e = lin(adapt_half, w, 1.0, nullptr, 0, nullptr, 0, nullptr, 0, -in_shift, st)) != cudaSuccess)
                    return cuda_fail(e, "bdf2 estimate store");
                x = adapt_full;
                y = adapt_half;
                n_it = std::max(i1.iters[0], it2);
            } else if (sdc) {
                // One SDC2 step from a fresh start.  Afterwards w holds level [1] and sdc_w0
                // level [0], both in the stored variable, whose difference is that of u.
                have_sdc = false;
                molt_status s1 = step(adapt_half, dt, MOLT_SDC2, st, &i1);
                if (s1 != MOLT_OK && s1 != MOLT_ERR_NOT_CONVERGED) return s1;
                x = w;
                y = sdc_w0;
                n_it = std::max(i1.iters[0], i1.iters[1]);
            } else {
                molt_status s1 = step(adapt_full, dt, MOLT_BE, st, &i1);
                molt_status s2 = step(adapt_half, 0.5 * dt, MOLT_BE, st, &i2);
                molt_status s3 = step(adapt_half, 0.5 * dt, MOLT_BE, st, &i3);
                for (molt_status s : {s1, s2, s3})
                    if (s != MOLT_OK && s != MOLT_ERR_NOT_CONVERGED) return s;
                x = adapt_full;
                y = adapt_half;
                n_it = std::max({i1.iters[0], i2.iters[0], i3.iters[0]});
            }
            if ((e = molt::max_abs_diff<T>(x, y, static_cast<long long>(count()), red, st)) != cudaSuccess ||
                (e = cudaMemcpyAsync(red_host, red, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st)) !=
                    cudaSuccess ||
                (e = cudaStreamSynchronize(st)) != cudaSuccess)
                return cuda_fail(e, "adaptive estimate");
            double diff;
            std::memcpy(&diff, &red_host[0], sizeof(double));
            const double eta = (sdc || bdf) ? diff : 0.5 * diff;   // the factor 1/2 is Richardson's
            double next;
            const bool ok = step_size_rule(eta, n_it, dt, a, &next, p.max_iter);
            if (ok) {
                if (want_bdf && (e = lin(adapt_prev, u, 1.0, nullptr, 0, nullptr, 0, nullptr, 0, 0, st)) != cudaSuccess)
                    return cuda_fail(e, "adaptive history");
                if ((e = lin(u, adapt_half, 1.0, nullptr, 0, nullptr, 0, nullptr, 0, 0, st)) != cudaSuccess)
                    return cuda_fail(e, "adaptive store");
                have_adapt_prev = want_bdf;
                dt_adapt_prev = dt;
                have_prev = have_prev2 = have_sdc = false;
                if (out) {
                    out->dt_used = dt;
                    out->dt_next = next;
                    out->eta = eta;
                    out->rejections = rejections;
                    out->max_iters = n_it;
                }
                return MOLT_OK;
            }
            ++rejections;
            if (dt <= a.dt_min) {
                have_prev = have_prev2 = have_sdc = false;
                return fail(MOLT_ERR_NOT_CONVERGED, "adaptive step: dt_min reached without meeting the LTE tolerance");
            }
            dt = next;
        }
    }

    // Vector CH step (Sec. 5.2) on the two device fields u1, u2 in place, in the stored variable
    // v = u - z3, z3 = (-1/2, -sqrt(3)/2).  BE, or BDF2 (Eq. BDF2 per component) with a BE start
    // that is repeated whenever dt changes.
    molt_status vch_step(void* u1v, void* u2v, double dt, int scheme, cudaStream_t st,
                         molt_step_info* info) override {
        T* u1 = static_cast<T*>(u1v);
        T* u2 = static_cast<T*>(u2v);
        if (info) std::memset(info, 0, sizeof(*info));
        if (scheme != MOLT_BE && scheme != MOLT_BDF2)
            return fail(MOLT_ERR_UNSUPPORTED, "vector CH steps support BE and BDF2");
        if (g.dim == 2 && g.nx > molt::max_row_length<T>(2))
            return fail(MOLT_ERR_UNSUPPORTED, "2D steps need x lines within the two-field row kernels' length");
        if (!vw2) {
            T** fields[] = {&vw2, &vY2, &vn2, &vp2, &vr2, &vg4, &vg5, &vg6, &vp1};
            for (T** f : fields)
                if (!alloc(f, count())) return fail(MOLT_ERR_OOM, "vector CH workspace");
        }
        const double zx = -0.5, zy = -0.86602540378443864676;
        cudaError_t e;
        if ((e = lin(w, u1, 1.0, nullptr, 0, nullptr, 0, nullptr, 0, -zx, st)) != cudaSuccess ||
            (e = lin(vw2, u2, 1.0, nullptr, 0, nullptr, 0, nullptr, 0, -zy, st)) != cudaSuccess ||
            (e = lin(wn, w, 1.0, nullptr, 0, nullptr, 0, nullptr, 0, 0, st)) != cudaSuccess ||
            (e = lin(vn2, vw2, 1.0, nullptr, 0, nullptr, 0, nullptr, 0, 0, st)) != cudaSuccess)
            return cuda_fail(e, "vector CH load");
        const bool bdf = scheme == MOLT_BDF2 && vch_have_prev && vch_dt_prev == dt;
        const T* r1 = wn;
        const T* r2 = vn2;
        double tau = dt;
        if (bdf) {
            tau = 2.0 * dt / 3.0;
            if ((e = lin(r, wn, 4.0 / 3.0, vp1, -1.0 / 3.0, nullptr, 0, nullptr, 0, 0, st)) != cudaSuccess ||
                (e = lin(vr2, vn2, 4.0 / 3.0, vp2, -1.0 / 3.0, nullptr, 0, nullptr, 0, 0, st)) != cudaSuccess)
                return cuda_fail(e, "vector CH bdf2 rhs");
            r1 = r;
            r2 = vr2;
        }
        Passes ps;
        double c_in, c_out;
        if (!make_vch_passes(tau, &ps, &c_in, &c_out)) return MOLT_ERR_ARG;
        if ((e = mm_inv(c_in, r1, f2, st)) != cudaSuccess || (e = mm_inv(c_out, f2, Y, st)) != cudaSuccess ||
            (e = mm_inv(c_in, r2, f2, st)) != cudaSuccess || (e = mm_inv(c_out, f2, vY2, st)) != cudaSuccess)
            return cuda_fail(e, "vector CH rhs inverse");
        int it;
        double res, tu;
        molt_status ms = stage(tau, nullptr, st, &it, &res, &tu, true, &ps);
        if (ms != MOLT_OK && ms != MOLT_ERR_NOT_CONVERGED) return ms;
        record(info, 0, it, res, tu);
        std::swap(vp1, wn);   // v^n becomes the previous level
        std::swap(vp2, vn2);
        vch_have_prev = true;
        vch_adapt_have_prev = false;
        vch_dt_prev = dt;
        if ((e = lin(u1, w, 1.0, nullptr, 0, nullptr, 0, nullptr, 0, zx, st)) != cudaSuccess ||
            (e = lin(u2, vw2, 1.0, nullptr, 0, nullptr, 0, nullptr, 0, zy, st)) != cudaSuccess)
            return cuda_fail(e, "vector CH store");
        if (info) info->status = ms;
        return ms;
    }

    // Vector CH: one stage solve v - tau F(v) = a_n v^n + a_p v^{n-1} for both components, from the
    // state (u1, u2) (also the first guess) and the optional earlier state (p1, p2), all in the
    // physical variable u; the result goes to (o1, o2), which may alias (u1, u2).
    T *va1 = nullptr, *va2 = nullptr, *vb1 = nullptr, *vb2 = nullptr, *vq1 = nullptr, *vq2 = nullptr;
    molt_status vch_stage_from(const T* u1, const T* u2, double an, const T* p1, const T* p2, double ap, double tau,
                               T* o1, T* o2, cudaStream_t st, int* iters) {
        const double zx = -0.5, zy = -0.86602540378443864676;
        cudaError_t e;
        if ((e = lin(w, u1, 1.0, nullptr, 0, nullptr, 0, nullptr, 0, -zx, st)) != cudaSuccess ||
            (e = lin(vw2, u2, 1.0, nullptr, 0, nullptr, 0, nullptr, 0, -zy, st)) != cudaSuccess ||
            (e = lin(r, u1, an, p1, p1 ? ap : 0.0, nullptr, 0, nullptr, 0, -zx * (an + (p1 ? ap : 0.0)), st)) !=
                cudaSuccess ||
            (e = lin(vr2, u2, an, p2, p2 ? ap : 0.0, nullptr, 0, nullptr, 0, -zy * (an + (p2 ? ap : 0.0)), st)) !=
                cudaSuccess)
            return cuda_fail(e, "vector stage load");
        Passes ps;
        double c_in, c_out;
        if (!make_vch_passes(tau, &ps, &c_in, &c_out)) return MOLT_ERR_ARG;
        if ((e = mm_inv(c_in, r, f2, st)) != cudaSuccess || (e = mm_inv(c_out, f2, Y, st)) != cudaSuccess ||
            (e = mm_inv(c_in, vr2, f2, st)) != cudaSuccess || (e = mm_inv(c_out, f2, vY2, st)) != cudaSuccess)
            return cuda_fail(e, "vector stage rhs inverse");
        double res, tu;
        molt_status ms = stage(tau, nullptr, st, iters, &res, &tu, true, &ps);
        if (ms != MOLT_OK && ms != MOLT_ERR_NOT_CONVERGED) return ms;
        if ((e = lin(o1, w, 1.0, nullptr, 0, nullptr, 0, nullptr, 0, zx, st)) != cudaSuccess ||
            (e = lin(o2, vw2, 1.0, nullptr, 0, nullptr, 0, nullptr, 0, zy, st)) != cudaSuccess)
            return cuda_fail(e, "vector stage store");
        return MOLT_OK;
    }

    double max_diff(const T* a, const T* b, cudaStream_t st, cudaError_t* err) {
        double v = 0.0;
        if ((*err = molt::max_abs_diff<T>(a, b, static_cast<long long>(count()), red, st)) != cudaSuccess ||
            (*err = cudaMemcpyAsync(red_host, red, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st)) !=
                cudaSuccess ||
            (*err = cudaStreamSynchronize(st)) != cudaSuccess)
            return 0.0;
        std::memcpy(&v, &red_host[0], sizeof(double));
        return v;
    }

    // Algorithm 1 (Sec. 5) for the vector model, as Sec. 6.2.2 runs it: the Richardson estimate of
    // BE, or BE-BDF2 with the variable-step BDF2 of the scalar controller; without history (the
    // first step) BE-BDF2 takes the Richardson estimate (the vector model has no SDC2 here).
    molt_status vch_adaptive(void* u1v, void* u2v, double dt, const molt_adaptive& a, cudaStream_t st,
                             molt_adaptive_info* out) override {
        T* u1 = static_cast<T*>(u1v);
        T* u2 = static_cast<T*>(u2v);
        if (a.estimator != MOLT_LTE_RICHARDSON && a.estimator != MOLT_LTE_BDF2)
            return fail(MOLT_ERR_UNSUPPORTED, "vector adaptive steps support the Richardson and BE-BDF2 estimates");
        if (g.dim == 2 && g.nx > molt::max_row_length<T>(2))
            return fail(MOLT_ERR_UNSUPPORTED, "2D steps need x lines within the two-field row kernels' length");
        if (!vw2) {
            T** fields[] = {&vw2, &vY2, &vn2, &vp2, &vr2, &vg4, &vg5, &vg6, &vp1};
            for (T** f : fields)
                if (!alloc(f, count())) return fail(MOLT_ERR_OOM, "vector CH workspace");
        }
        if (!va1) {
            T** fields[] = {&va1, &va2, &vb1, &vb2, &vq1, &vq2};
            for (T** f : fields)
                if (!alloc(f, count())) return fail(MOLT_ERR_OOM, "vector adaptive workspace");
        }
        const bool want_bdf = a.estimator == MOLT_LTE_BDF2;
        cudaError_t e = cudaSuccess;
        int rejections = 0;
        for (;;) {
            const bool bdf = want_bdf && vch_adapt_have_prev;
            int n_it = 0, it;
            molt_status ms;
            double diff;
            if (bdf) {
                // BE into (va), variable-step BDF2 into (vb) from the same start
                if ((ms = vch_stage_from(u1, u2, 1.0, nullptr, nullptr, 0.0, dt, va1, va2, st, &it)) != MOLT_OK &&
                    ms != MOLT_ERR_NOT_CONVERGED)
                    return ms;
                n_it = it;
                const double om = dt / vch_adapt_dt_prev;
                const double tau = dt * (1.0 + om) / (1.0 + 2.0 * om);
                const double an = (1.0 + om) * (1.0 + om) / (1.0 + 2.0 * om), ap = -om * om / (1.0 + 2.0 * om);
                if ((ms = vch_stage_from(u1, u2, an, vq1, vq2, ap, tau, vb1, vb2, st, &it)) != MOLT_OK &&
                    ms != MOLT_ERR_NOT_CONVERGED)
                    return ms;
                n_it = std::max(n_it, it);
                diff = std::max(max_diff(vb1, va1, st, &e), e == cudaSuccess ? max_diff(vb2, va2, st, &e) : 0.0);
            } else {
                // one BE step into (va), two half steps into (vb)
                if ((ms = vch_stage_from(u1, u2, 1.0, nullptr, nullptr, 0.0, dt, va1, va2, st, &it)) != MOLT_OK &&
                    ms != MOLT_ERR_NOT_CONVERGED)
                    return ms;
                n_it = it;
                if ((ms = vch_stage_from(u1, u2, 1.0, nullptr, nullptr, 0.0, 0.5 * dt, vb1, vb2, st, &it)) != MOLT_OK &&
                    ms != MOLT_ERR_NOT_CONVERGED)
                    return ms;
                n_it = std::max(n_it, it);
                if ((ms = vch_stage_from(vb1, vb2, 1.0, nullptr, nullptr, 0.0, 0.5 * dt, vb1, vb2, st, &it)) !=
                        MOLT_OK &&
                    ms != MOLT_ERR_NOT_CONVERGED)
                    return ms;
                n_it = std::max(n_it, it);
                diff = std::max(max_diff(va1, vb1, st, &e), e == cudaSuccess ? max_diff(va2, vb2, st, &e) : 0.0);
            }
            if (e != cudaSuccess) return cuda_fail(e, "vector adaptive estimate");
            const double eta = bdf ? diff : 0.5 * diff;   // the factor 1/2 is Richardson's
            double next;
            const bool ok = step_size_rule(eta, n_it, dt, a, &next, p.max_iter);
            if (ok) {
                if (want_bdf && ((e = lin(vq1, u1, 1.0, nullptr, 0, nullptr, 0, nullptr, 0, 0, st)) != cudaSuccess ||
                                 (e = lin(vq2, u2, 1.0, nullptr, 0, nullptr, 0, nullptr, 0, 0, st)) != cudaSuccess))
                    return cuda_fail(e, "vector adaptive history");
                if ((e = lin(u1, vb1, 1.0, nullptr, 0, nullptr, 0, nullptr, 0, 0, st)) != cudaSuccess ||
                    (e = lin(u2, vb2, 1.0, nullptr, 0, nullptr, 0, nullptr, 0, 0, st)) != cudaSuccess)
                    return cuda_fail(e, "vector adaptive store");
                vch_adapt_have_prev = want_bdf;
                vch_adapt_dt_prev = dt;
                vch_have_prev = false;
                if (out) {
                    out->dt_used = dt;
                    out->dt_next = next;
                    out->eta = eta;
                    out->rejections = rejections;
                    out->max_iters = n_it;
                }
                return MOLT_OK;
            }
            ++rejections;
            if (dt <= a.dt_min)
                return fail(MOLT_ERR_NOT_CONVERGED, "adaptive step: dt_min reached without meeting the LTE tolerance");
            dt = next;
        }
    }

    molt_status apply(int axis, double c, const void* in, void* out, cudaStream_t st) override {
        if (axis != 0 && axis != 1) return fail(MOLT_ERR_ARG, "axis must be 0 (x) or 1 (y)");
        if (axis == 1 && g.dim != 2) return fail(MOLT_ERR_ARG, "axis 1 needs a 2D grid");
        if (axis == 1 && in == out) return fail(MOLT_ERR_ARG, "column sweeps cannot run in place");
        if (!(c > 0.0) || !std::isfinite(c)) return fail(MOLT_ERR_ARG, "c must be positive and finite");
        molt::LineParams<T> lp;
        if (!line_params(c, axis, &lp)) return MOLT_ERR_ARG;
        cudaError_t e = copy_sweep(axis, lp, static_cast<const T*>(in), static_cast<T*>(out), st);
        if (e != cudaSuccess) return cuda_fail(e, "sweep");
        return MOLT_OK;
    }

    molt_status apply_tc(double c, const void* in, void* out, cudaStream_t st) override {
        if (!fp32() || bc != molt::BC_PERIODIC || !molt::rows_tc_supported(g.nx, g.ny, p.quad_order))
            return fail(MOLT_ERR_UNSUPPORTED, "tensor-core row sweeps need FP32, periodic lines of 1024..8192 nodes "
                                              "(a power of two) and a multiple of 8192/nx lines");
        if (!(c > 0.0) || !std::isfinite(c)) return fail(MOLT_ERR_ARG, "c must be positive and finite");
        if (in == out) return fail(MOLT_ERR_ARG, "tensor-core row sweeps cannot run in place");
        const cudaError_t e = tc_sweep(c, static_cast<const T*>(in), static_cast<T*>(out), st);
        if (e == cudaErrorNotReady) return fail(MOLT_ERR_UNSUPPORTED, "operands are not built during stream capture");
        if (e != cudaSuccess) return cuda_fail(e, "tensor-core row sweep");
        return MOLT_OK;
    }

    // The autotuner (molt_autotune): times every available launch of each sweep of a step on this
    // grid and keeps the fastest.  Test data: hash-uniform fields in [-0.5, 0.5).
    molt_status autotune(cudaStream_t st, molt_tuning* out, int capacity, int* nout) override {
        *nout = 0;
        if (!fp32()) return MOLT_OK;   // FP64 sweeps have one kernel family
        cudaError_t e;
        T* fl[7] = {w, f1, f2, f3, f4, f5, f6};
        for (int k = 0; k < 7; ++k)
            if ((e = molt::fill_pattern<T>(fl[k], static_cast<long long>(count()), 11u + k, -0.5, 0.5, st)) !=
                cudaSuccess)
                return cuda_fail(e, "autotune data");
        if ((e = molt::fill_pattern<T>(Y, static_cast<long long>(count()), 7u, -0.5, 0.5, st)) != cudaSuccess)
            return cuda_fail(e, "autotune data");
        const double hx = grid_h(g.nx, g.Lx, bc), hy = g.dim == 2 ? grid_h(g.ny, g.Ly, bc) : hx;
        const double cx = (hx / 0.3) * (hx / 0.3), cy = (hy / 0.3) * (hy / 0.3);
        molt::LineParams<T> lx, ly;
        if (!line_params(cx, 0, &lx) || (g.dim == 2 && !line_params(cy, 1, &ly))) return MOLT_ERR_ARG;
        const StageParams sp = stage_params(1e-3, p.eps);
        Passes ps, pv;
        double vc_in = 0.0, vc_out = 0.0;
        if (!make_passes(sp, &ps) || !make_vch_passes(1e-3, &pv, &vc_in, &vc_out)) return MOLT_ERR_ARG;
        // the vector passes are timed on the scalar work fields (f6 stands in for the second
        // component), so tuning needs no vector workspace
        struct Entry { int pass, kind, axis; };
        static const Entry k2d[] = {{0, molt::OP_COPY, 0}, {0, molt::OP_COPY, 1}, {1, molt::OP_P1, 1},
                                    {2, molt::OP_P2, 0},   {3, molt::OP_P3, 1},   {4, molt::OP_P4, 0},
                                    {7, molt::OP_V1, 1},   {8, molt::OP_V2, 0}};
        static const Entry k1d[] = {{0, molt::OP_COPY, 0}, {5, molt::OP_1A, 0}, {6, molt::OP_1B, 0},
                                    {9, molt::OP_V1A, 0}};
        const Entry* ebeg = g.dim == 2 ? k2d : k1d;
        const Entry* eend = g.dim == 2 ? k2d + 8 : k1d + 4;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
            if (e0) cudaEventDestroy(e0);
            return fail(MOLT_ERR_CUDA, "autotune events");
        }
        molt_status result = MOLT_OK;
        for (const Entry* ep = ebeg; ep != eend; ++ep) {
            const Entry& en = *ep;
            molt::OpArgs<T> a;
            a.g2 = ps.g2;
            a.g1 = ps.g1;
            a.beta = ps.beta;
            a.shift = ps.s;
            switch (en.kind) {
                case molt::OP_COPY: a.in0 = f1; a.out0 = f2; break;
                case molt::OP_P1: a.in0 = w; a.out0 = f1; a.out1 = f2; break;
                case molt::OP_P2: a.in0 = w; a.in1 = f1; a.in2 = f2; a.out0 = f3; a.out1 = f4; break;
                case molt::OP_P3: a.in0 = f3; a.in1 = f4; a.out0 = f5; a.out1 = f6; break;
                case molt::OP_P4: a.in0 = f5; a.in1 = f6; a.in2 = f4; a.in3 = Y; a.out0 = f1; break;
                case molt::OP_1A: a.in0 = w; a.out0 = f1; break;
                case molt::OP_V1: a.in0 = w; a.in1 = f6; a.out0 = f1; a.out1 = f2; break;
                case molt::OP_V2: a.in0 = w; a.in1 = f6; a.in2 = f1; a.in3 = f2; a.out0 = f3; a.out1 = f4; break;
                case molt::OP_V1A: a.in0 = w; a.in1 = f6; a.out0 = f1; break;
                default: a.in0 = f1; a.in1 = Y; a.out0 = f2; break;   // OP_1B
            }
            if (en.kind == molt::OP_V1 || en.kind == molt::OP_V2 || en.kind == molt::OP_V1A) {
                a.vs = pv.vs;
                a.beta = pv.beta;
                a.comp = 0;
            }
            const molt::LineParams<T>& lp = en.axis == 0 ? lx : ly;
            std::vector<int> cand = en.axis == 0
                ? std::vector<int>{molt::LAUNCH_ROWS_ONE_BLOCK, molt::LAUNCH_ROWS_CLUSTER2, molt::LAUNCH_ROWS_GENERAL}
                : std::vector<int>{molt::LAUNCH_COLS_TMA, molt::LAUNCH_COLS_CP_ASYNC, molt::LAUNCH_COLS_GENERAL};
            const bool tc_ok = en.kind == molt::OP_COPY && en.axis == 0 && bc == molt::BC_PERIODIC &&
                               molt::rows_tc_supported(g.nx, g.ny, p.quad_order);
            if (tc_ok) cand.push_back(molt::LAUNCH_ROWS_TENSOR_CORE);
            molt_tuning rec{};
            rec.pass = en.pass;
            rec.axis = en.axis;
            rec.candidates = static_cast<int>(cand.size());
            double best = INFINITY;
            int chosen = 0;
            for (size_t ci = 0; ci < cand.size(); ++ci) {
                rec.launch[ci] = cand[ci];
                rec.ms[ci] = -1.0;
                auto run = [&]() -> cudaError_t {
                    if (cand[ci] == molt::LAUNCH_ROWS_TENSOR_CORE) return tc_sweep(cx, a.in0, a.out0, st);
                    molt::OpArgs<T> b = a;
                    b.variant = cand[ci];
                    return molt::sweep<T>(en.axis, lp, en.kind, b, g.nx, g.ny, &cs, red, st, nullptr, nullptr);
                };
                if (run() != cudaSuccess) {            // not available for this grid
                    cudaGetLastError();
                    continue;
                }
                float ms = 0.0f;
                constexpr int reps = 5;
                if ((e = cudaEventRecord(e0, st)) != cudaSuccess) break;
                for (int r = 0; r < reps && e == cudaSuccess; ++r) e = run();
                if (e != cudaSuccess || (e = cudaEventRecord(e1, st)) != cudaSuccess ||
                    (e = cudaEventSynchronize(e1)) != cudaSuccess || (e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess)
                    break;
                double per = static_cast<double>(ms) / reps;
                if (cand[ci] == molt::LAUNCH_ROWS_TENSOR_CORE) {
                    // kept only where it is as accurate as the FP32 sweep bar: 1e-6 of max|H f|
                    molt::OpArgs<T> b = a;
                    b.out0 = f3;
                    double dref = 0.0, dmax = 0.0;
                    if ((e = molt::sweep<T>(0, lp, molt::OP_COPY, b, g.nx, g.ny, &cs, red, st, nullptr, nullptr)) !=
                            cudaSuccess ||
                        (e = molt::fill_pattern<T>(f5, static_cast<long long>(count()), 0u, 0.0, 0.0, st)) != cudaSuccess)
                        break;
                    dmax = max_diff(f2, f3, st, &e);
                    if (e == cudaSuccess) dref = max_diff(f3, f5, st, &e);
                    if (e != cudaSuccess) break;
                    rec.tc_rel_diff = dmax / dref;
                    if (!(dmax <= 1e-6 * dref)) per = -per;   // recorded, not eligible
                }
                rec.ms[ci] = per;
                if (per > 0.0 && per < best) {
                    best = per;
                    chosen = cand[ci];
                }
            }
            if (e != cudaSuccess) {
                result = cuda_fail(e, "autotune");
                break;
            }
            rec.chosen = chosen;
            tune[en.kind][en.axis] = chosen;
            if (*nout < capacity && out) out[*nout] = rec;
            ++*nout;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaMemsetAsync(red, 0, 2 * sizeof(unsigned long long), st);
        drop_graphs();   // graphs captured the previous choices
        have_prev = have_prev2 = have_sdc = have_adapt_prev = vch_have_prev = vch_adapt_have_prev = false;
        return result;
    }
};

molt_status validate_params(const molt_grid* g, const molt_params* p, std::string* m) {
    if (!p) { *m = "null parameters"; return MOLT_ERR_ARG; }
    if (!(p->eps > 0.0) || !std::isfinite(p->eps)) { *m = "eps must be positive"; return MOLT_ERR_ARG; }
    if (p->quad_order != 2 && p->quad_order != 4 && p->quad_order != 6) { *m = "quad_order must be 2, 4 or 6"; return MOLT_ERR_ARG; }
    if (p->precision != MOLT_FP32 && p->precision != MOLT_FP64) { *m = "unknown precision"; return MOLT_ERR_ARG; }
    if (!(p->tol > 0.0)) { *m = "tol must be positive"; return MOLT_ERR_ARG; }
    if (p->max_iter < 1) { *m = "max_iter must be >= 1"; return MOLT_ERR_ARG; }
    const int minn = p->quad_order + 2;
    if (g->nx < minn || (g->dim == 2 && g->ny < minn)) { *m = "grid lines too short for the quadrature order"; return MOLT_ERR_ARG; }
    const int maxn = p->precision == MOLT_FP32 ? molt::max_row_length<float>(1) : molt::max_row_length<double>(1);
    if (g->nx > maxn) { *m = "x lines longer than the row kernels support"; return MOLT_ERR_ARG; }
    return MOLT_OK;
}

molt_status set_global_error(molt_status s, const char* m) {
    g_last_error = m;
    return s;
}

}  // namespace

void molt::set_abi_error(const char* message) { g_last_error = message ? message : ""; }
void molt::count_tma_launch() { g_tma_launches.fetch_add(1); }

extern "C" {

molt_status molt_grid_create(molt_grid** grid, int dim, int nx, int ny, double Lx, double Ly, int bc) {
    if (!grid) return set_global_error(MOLT_ERR_ARG, "null grid pointer");
    *grid = nullptr;
    if (dim != 1 && dim != 2) return set_global_error(MOLT_ERR_ARG, "dim must be 1 or 2");
    if (dim == 1 && ny != 1) return set_global_error(MOLT_ERR_ARG, "1D grids need ny = 1");
    if (nx < 8 || (dim == 2 && ny < 8)) return set_global_error(MOLT_ERR_ARG, "each direction needs at least 8 nodes");
    if (!(Lx > 0.0) || (dim == 2 && !(Ly > 0.0))) return set_global_error(MOLT_ERR_ARG, "domain lengths must be positive");
    if (bc < MOLT_BC_PERIODIC || bc > MOLT_BC_DIRICHLET) return set_global_error(MOLT_ERR_ARG, "unknown boundary condition");
    if (static_cast<long long>(nx) * ny > (1LL << 31) - 1) return set_global_error(MOLT_ERR_ARG, "grid too large");
    molt_grid* g = new (std::nothrow) molt_grid{dim, nx, ny, Lx, dim == 2 ? Ly : 1.0, bc};
    if (!g) return set_global_error(MOLT_ERR_OOM, "host allocation failed");
    *grid = g;
    return MOLT_OK;
}

void molt_grid_destroy(molt_grid* grid) { delete grid; }

molt_status molt_solver_create(molt_solver** solver, const molt_grid* grid, const molt_params* p) {
    if (!solver || !grid) return set_global_error(MOLT_ERR_ARG, "null argument");
    *solver = nullptr;
    std::string m;
    molt_status s = validate_params(grid, p, &m);
    if (s != MOLT_OK) return set_global_error(s, m.c_str());
    molt_solver* h = nullptr;
    if (p->precision == MOLT_FP32) h = new (std::nothrow) Solver<float>();
    else h = new (std::nothrow) Solver<double>();
    if (!h) return set_global_error(MOLT_ERR_OOM, "host allocation failed");
    h->g = *grid;
    h->p = *p;
    h->bc = grid->bc;
    cudaGetDevice(&h->device);
    s = h->init();
    if (s != MOLT_OK) {
        g_last_error = h->err;
        delete h;
        return s;
    }
    *solver = h;
    return MOLT_OK;
}

void molt_solver_destroy(molt_solver* solver) { delete solver; }

molt_status molt_set_params(molt_solver* s, const molt_params* p) {
    if (!s) return set_global_error(MOLT_ERR_ARG, "null solver");
    std::string m;
    molt_status st = validate_params(&s->g, p, &m);
    if (st != MOLT_OK) { s->err = m; return st; }
    if (p->precision != s->p.precision) { s->err = "precision cannot change"; return MOLT_ERR_ARG; }
    s->p = *p;
    s->have_prev = false;
    s->have_prev2 = false;
    s->have_sdc = false;
    s->have_adapt_prev = false;
    s->vch_have_prev = false;
    s->vch_adapt_have_prev = false;
    s->drop_graphs();
    return MOLT_OK;
}

molt_status molt_set_bc(molt_solver* s, int bc) {
    if (!s) return set_global_error(MOLT_ERR_ARG, "null solver");
    if (bc < MOLT_BC_PERIODIC || bc > MOLT_BC_DIRICHLET) { s->err = "unknown boundary condition"; return MOLT_ERR_ARG; }
    s->bc = bc;
    s->g.bc = bc;
    s->have_prev = false;
    s->have_prev2 = false;
    s->have_sdc = false;
    s->have_adapt_prev = false;
    s->vch_have_prev = false;
    s->vch_adapt_have_prev = false;
    s->drop_graphs();
    return MOLT_OK;
}

molt_status molt_set_execution(molt_solver* s, int mode) {
    if (!s) return set_global_error(MOLT_ERR_ARG, "null solver");
    if (mode != MOLT_EXEC_HOST_LOOP && mode != MOLT_EXEC_GRAPH) { s->err = "unknown execution mode"; return MOLT_ERR_ARG; }
    s->exec_mode = mode;
    return MOLT_OK;
}

long long molt_graph_fallbacks(const molt_solver* s) { return s ? s->graph_fallbacks : 0; }

molt_status molt_reset_history(molt_solver* s) {
    if (!s) return set_global_error(MOLT_ERR_ARG, "null solver");
    s->have_prev = false;
    s->have_prev2 = false;
    s->have_sdc = false;
    s->have_adapt_prev = false;
    s->vch_have_prev = false;
    s->vch_adapt_have_prev = false;
    return MOLT_OK;
}

molt_status molt_step(molt_solver* s, void* u_dev, double dt, int scheme, void* stream, molt_step_info* info) {
    if (!s) return set_global_error(MOLT_ERR_ARG, "null solver");
    if (!u_dev) { s->err = "null field"; return MOLT_ERR_ARG; }
    if (!(dt > 0.0) || !std::isfinite(dt)) { s->err = "dt must be positive"; return MOLT_ERR_ARG; }
    if (scheme < MOLT_BE || scheme > MOLT_BDF3) { s->err = "unknown scheme"; return MOLT_ERR_ARG; }
    s->have_adapt_prev = false;
    return s->step(u_dev, dt, scheme, static_cast<cudaStream_t>(stream), info);
}

molt_status molt_run_host(molt_solver* s, void* u_host, double dt, int scheme, int nsteps, void* stream,
                          molt_step_info* info) {
    if (!s) return set_global_error(MOLT_ERR_ARG, "null solver");
    if (!u_host || nsteps < 0) { s->err = "bad host buffer or step count"; return MOLT_ERR_ARG; }
    if (!(dt > 0.0) || !std::isfinite(dt)) { s->err = "dt must be positive"; return MOLT_ERR_ARG; }
    if (scheme < MOLT_BE || scheme > MOLT_BDF3) { s->err = "unknown scheme"; return MOLT_ERR_ARG; }
    s->have_adapt_prev = false;
    return s->run_host(u_host, dt, scheme, nsteps, static_cast<cudaStream_t>(stream), info);
}

molt_status molt_energy(molt_solver* s, const void* u_dev, double* energy, void* stream) {
    if (!s) return set_global_error(MOLT_ERR_ARG, "null solver");
    if (!u_dev || !energy) { s->err = "null argument"; return MOLT_ERR_ARG; }
    return s->reduce(u_dev, 0, energy, static_cast<cudaStream_t>(stream));
}

molt_status molt_mass(molt_solver* s, const void* u_dev, double* mass, void* stream) {
    if (!s) return set_global_error(MOLT_ERR_ARG, "null solver");
    if (!u_dev || !mass) { s->err = "null argument"; return MOLT_ERR_ARG; }
    return s->reduce(u_dev, 1, mass, static_cast<cudaStream_t>(stream));
}

molt_status molt_helmholtz_apply(molt_solver* s, int axis, double c, const void* in_dev, void* out_dev, void* stream) {
    if (!s) return set_global_error(MOLT_ERR_ARG, "null solver");
    if (!in_dev || !out_dev) { s->err = "null field"; return MOLT_ERR_ARG; }
    return s->apply(axis, c, in_dev, out_dev, static_cast<cudaStream_t>(stream));
}

molt_status molt_vch_step_adaptive(molt_solver* s, void* u1, void* u2, double dt, const molt_adaptive* a,
                                   void* stream, molt_adaptive_info* info) {
    if (!s) return set_global_error(MOLT_ERR_ARG, "null solver");
    if (!u1 || !u2 || u1 == u2 || !a) { s->err = "null or equal fields, or null parameters"; return MOLT_ERR_ARG; }
    if (!(dt > 0.0) || !(a->lte_tol > 0.0) || !(a->dt_min > 0.0) || a->dt_max < a->dt_min || !(a->theta > 0.0) ||
        !(a->gamma > 1.0)) {
        s->err = "bad adaptive parameters";
        return MOLT_ERR_ARG;
    }
    return s->vch_adaptive(u1, u2, std::min(std::max(dt, a->dt_min), a->dt_max), *a, static_cast<cudaStream_t>(stream),
                           info);
}

molt_status molt_autotune(molt_solver* s, void* stream, molt_tuning* entries, int capacity, int* count) {
    if (!s) return set_global_error(MOLT_ERR_ARG, "null solver");
    int n = 0;
    const molt_status st = s->autotune(static_cast<cudaStream_t>(stream), entries, capacity < 0 ? 0 : capacity, &n);
    if (count) *count = n;
    return st;
}

molt_status molt_helmholtz_rows_tc(molt_solver* s, double c, const void* in_dev, void* out_dev, void* stream) {
    if (!s) return set_global_error(MOLT_ERR_ARG, "null solver");
    if (!in_dev || !out_dev) { s->err = "null field"; return MOLT_ERR_ARG; }
    return s->apply_tc(c, in_dev, out_dev, static_cast<cudaStream_t>(stream));
}

molt_status molt_quadrature_weights(double nu, int M, const int* offsets, int side, double* weights) {
    if (M != 2 && M != 4 && M != 6) return set_global_error(MOLT_ERR_ARG, "M must be 2, 4 or 6");
    if (side != 0 && side != 1) return set_global_error(MOLT_ERR_ARG, "side must be 0 (L) or 1 (R)");
    if (!molt::quadrature_weights(nu, M, offsets, side, weights)) return set_global_error(MOLT_ERR_ARG, "bad nu or pointer");
    return MOLT_OK;
}

const char* molt_last_error(const molt_solver* s) {
    if (!s) return g_last_error.c_str();
    return s->err.c_str();
}

molt_status molt_vch_step(molt_solver* s, void* u1_dev, void* u2_dev, double dt, int scheme, void* stream,
                          molt_step_info* info) {
    if (!s) return set_global_error(MOLT_ERR_ARG, "null solver");
    if (!u1_dev || !u2_dev || u1_dev == u2_dev) { s->err = "need two distinct component fields"; return MOLT_ERR_ARG; }
    if (!(dt > 0.0) || !std::isfinite(dt)) { s->err = "dt must be positive"; return MOLT_ERR_ARG; }
    if (scheme < MOLT_BE || scheme > MOLT_BDF3) { s->err = "unknown scheme"; return MOLT_ERR_ARG; }
    return s->vch_step(u1_dev, u2_dev, dt, scheme, static_cast<cudaStream_t>(stream), info);
}

molt_status molt_step_adaptive(molt_solver* s, void* u, double dt, const molt_adaptive* a, void* stream,
                               molt_adaptive_info* info) {
    if (!s) return set_global_error(MOLT_ERR_ARG, "null solver");
    if (!u || !a) {
        s->err = "null field or parameters";
        return MOLT_ERR_ARG;
    }
    if (!(dt > 0.0) || !(a->lte_tol > 0.0) || !(a->dt_min > 0.0) || !(a->dt_max >= a->dt_min) ||
        !(a->theta > 0.0) || !(a->gamma > 1.0) || !std::isfinite(dt) || !std::isfinite(a->dt_max) ||
        (a->estimator != MOLT_LTE_RICHARDSON && a->estimator != MOLT_LTE_SDC2 && a->estimator != MOLT_LTE_BDF2))
    {
        s->err = "adaptive parameters: need dt, lte_tol, dt_min > 0, dt_max >= dt_min, theta > 0, gamma > 1, "
                 "estimator MOLT_LTE_RICHARDSON, MOLT_LTE_SDC2 or MOLT_LTE_BDF2";
        return MOLT_ERR_ARG;
    }
    if (info) std::memset(info, 0, sizeof(*info));
    return s->adaptive(u, std::min(std::max(dt, a->dt_min), a->dt_max), *a, static_cast<cudaStream_t>(stream), info);
}

long long molt_kernel_launches(const molt_solver* s) { return s ? s->launches : 0; }

long long molt_column_tma_launches(void) { return g_tma_launches.load(); }

molt_status molt_profile_enable(molt_solver* s, int enable) {
    if (!s) return set_global_error(MOLT_ERR_ARG, "null solver");
    s->prof.on = enable != 0;
    return MOLT_OK;
}

molt_status molt_profile_collect(molt_solver* s, double* ms, long long* launches) {
    if (!s) return set_global_error(MOLT_ERR_ARG, "null solver");
    if (!ms || !launches) { s->err = "null output"; return MOLT_ERR_ARG; }
    cudaError_t e = s->prof.collect(ms, launches);
    if (e != cudaSuccess) { s->err = std::string("profile: ") + cudaGetErrorString(e); return MOLT_ERR_CUDA; }
    return MOLT_OK;
}

}  // extern "C"
