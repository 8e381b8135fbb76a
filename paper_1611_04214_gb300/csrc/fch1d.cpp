// The sixth-order (functionalized) Cahn-Hilliard model of the paper's last section on independent
// 1D lines, BE steps (Eq. FCH0 / FCH, completing the cube of Eq. FCH_BE with the PDE's signs).
//
// With a = (dt eps^4)^(1/3), H = (I - a Lap)^{-1} (the line inverse of Sec. 3 with c = a) and
// D = H - I, H Lap = D / a turns the lagged iteration
//   v^{k+1} = H^3 [v^n + dt Lap g(v^k) - (3a Lap - 3a^2 Lap^2) v^k],
//   g = -eps^2 Lap f - eps^2 f' Lap v + f f' + eta eps^4 Lap v - eta eps^2 f,
// into line sweeps with no explicit derivative:
//   v^{k+1} = H z,  z = H^2 v^n + (3 + c_eta) D^2 v - 3 H D v - c_f D^2 f + c_p H D p,
//   c_eta = dt eta eps^4 / a^2, c_f = dt eps^2 / a^2, c_p = dt / a,
//   p = -eps^2 f' Lap v + f f' - eta eps^2 f.
// Lap v^{k+1} = (v^{k+1} - z) / a holds exactly for the discrete H and is carried with the iterate
// (across steps too); initial data take Lap(H v^n) = (H v^n - v^n) / a for the first iteration.
// Each iteration is 7 line sweeps, one pointwise kernel and six linear combinations over the
// [lines][nx] field.  The stopping rule is the single-grid solver's
// (FP32: the tolerance floored at 2 ulp of max|v| and the stall rule below 64 ulp).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <initializer_list>
#include <string>
#include <vector>

#include "../../include/molt.h"
#include "molt_internal.h"

struct molt_fch1d {
    virtual ~molt_fch1d() = default;
    virtual molt_status step(void* u, double dt, cudaStream_t st, molt_step_info* info) = 0;
    long long launches = 0;
};

namespace {

molt_status fail_f(molt_status s, const std::string& m) {
    molt::set_abi_error(m.c_str());
    return s;
}

template <typename T>
struct Fch1d final : molt_fch1d {
    int nx = 0, lines = 0, bc = 0;
    double L = 0.0, eta = 0.0;
    molt_params p{};
    size_t n = 0;
    std::vector<void*> allocs;
    T *v = nullptr, *vn = nullptr, *vnew = nullptr, *h2vn = nullptr, *lap = nullptr, *f = nullptr, *pp = nullptr;
    T *hv = nullptr, *dv = nullptr, *hdv = nullptr, *df = nullptr, *hdf = nullptr, *dp = nullptr, *hdp = nullptr,
      *z = nullptr, *zero = nullptr;
    molt::ColScratch<T> cs{};   // unused by row sweeps
    unsigned long long* red = nullptr;
    unsigned long long* red_host = nullptr;
    bool have_lap = false;   // Lap v of the last step's iterate is in `lap`

    ~Fch1d() override {
        for (void* q : allocs) cudaFree(q);
        if (red_host) cudaFreeHost(red_host);
    }

    bool alloc(T** q) {
        void* m = nullptr;
        if (cudaMalloc(&m, n * sizeof(T)) != cudaSuccess) return false;
        allocs.push_back(m);
        *q = static_cast<T*>(m);
        return true;
    }

    bool init() {
        for (T** q : {&v, &vn, &vnew, &h2vn, &lap, &f, &pp, &hv, &dv, &hdv, &df, &hdf, &dp, &hdp, &z, &zero})
            if (!alloc(q)) return false;
        void* m = nullptr;
        if (cudaMalloc(&m, 2 * sizeof(unsigned long long)) != cudaSuccess) return false;
        allocs.push_back(m);
        red = static_cast<unsigned long long*>(m);
        return cudaMemset(zero, 0, n * sizeof(T)) == cudaSuccess &&
               cudaMallocHost(&red_host, 2 * sizeof(unsigned long long)) == cudaSuccess;
    }

    cudaError_t H(const molt::LineParams<T>& lp, const T* in, T* out, cudaStream_t st) {
        molt::OpArgs<T> a;
        a.in0 = in;
        a.out0 = out;
        return molt::sweep<T>(0, lp, molt::OP_COPY, a, nx, lines, &cs, red, st, &launches);
    }

    cudaError_t lin(T* out, const T* x0, double c0, const T* x1, double c1, const T* x2, double c2, const T* x3,
                    double c3, double c4, cudaStream_t st) {
        return molt::lincomb<T>(out, static_cast<long long>(n), x0, c0, x1, c1, x2, c2, x3, c3, c4, st, &launches);
    }

    double read_max(const T* a, const T* b, cudaStream_t st, cudaError_t* e) {
        double r = 0.0;
        if ((*e = molt::max_abs_diff<T>(a, b, static_cast<long long>(n), red, st)) != cudaSuccess ||
            (*e = cudaMemcpyAsync(red_host, red, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st)) !=
                cudaSuccess ||
            (*e = cudaStreamSynchronize(st)) != cudaSuccess)
            return 0.0;
        std::memcpy(&r, red_host, sizeof(double));
        launches += 1;
        return r;
    }

    molt_status step(void* uv, double dt, cudaStream_t st, molt_step_info* info) override {
        T* u = static_cast<T*>(uv);
        const double eps = p.eps;
        const double a = std::cbrt(dt * eps * eps * eps * eps);
        const double c_eta = dt * eta * std::pow(eps, 4) / (a * a), c_f = dt * eps * eps / (a * a), c_p = dt / a;
        molt::LineParams<double> lpd;
        const char* err = nullptr;
        if (!molt::build_line_params(a, molt::grid_h(nx, L, bc), nx, p.quad_order, bc, &lpd, &err))
            return fail_f(MOLT_ERR_ARG, err ? err : "bad line parameters");
        const molt::LineParams<T> lp = molt::cast_line_params<T>(lpd);
        cudaError_t e;
        // v^n = u + 1; H^2 v^n; Lap v^n carried or bootstrapped
        if ((e = lin(vn, u, 1.0, nullptr, 0, nullptr, 0, nullptr, 0, 1.0, st)) != cudaSuccess ||
            (e = lin(v, vn, 1.0, nullptr, 0, nullptr, 0, nullptr, 0, 0.0, st)) != cudaSuccess ||
            (e = H(lp, vn, hv, st)) != cudaSuccess || (e = H(lp, hv, h2vn, st)) != cudaSuccess)
            return fail_f(MOLT_ERR_CUDA, std::string("sixth-order step load: ") + cudaGetErrorString(e));
        if (!have_lap)
            if ((e = lin(lap, hv, 1.0 / a, vn, -1.0 / a, nullptr, 0, nullptr, 0, 0.0, st)) != cudaSuccess)
                return fail_f(MOLT_ERR_CUDA, std::string("sixth-order step load: ") + cudaGetErrorString(e));
        double res = INFINITY, best = INFINITY, tol_used = p.tol;
        int k = 0, stall = 0;
        bool converged = false;
        const bool fp32 = sizeof(T) == 4;
        for (k = 1; k <= p.max_iter; ++k) {
            if ((e = molt::fch_pointwise<T>(static_cast<long long>(n), v, lap, eps * eps, eta * eps * eps, f, pp, st,
                                            &launches)) != cudaSuccess ||
                (e = H(lp, v, hv, st)) != cudaSuccess ||
                (e = lin(dv, hv, 1.0, v, -1.0, nullptr, 0, nullptr, 0, 0.0, st)) != cudaSuccess ||
                (e = H(lp, dv, hdv, st)) != cudaSuccess || (e = H(lp, f, hv, st)) != cudaSuccess ||
                (e = lin(df, hv, 1.0, f, -1.0, nullptr, 0, nullptr, 0, 0.0, st)) != cudaSuccess ||
                (e = H(lp, df, hdf, st)) != cudaSuccess || (e = H(lp, pp, hv, st)) != cudaSuccess ||
                (e = lin(dp, hv, 1.0, pp, -1.0, nullptr, 0, nullptr, 0, 0.0, st)) != cudaSuccess ||
                (e = H(lp, dp, hdp, st)) != cudaSuccess ||
                // z = H^2 v^n + c_eta H D v - (3 + c_eta) D v - c_f H D f + c_f D f + c_p H D p
                // (= ... + (3 + c_eta) D^2 v - 3 H D v - c_f D^2 f + c_p H D p with D^2 = H D - D)
                (e = lin(z, h2vn, 1.0, hdv, c_eta, dv, -(3.0 + c_eta), hdf, -c_f, 0.0, st)) != cudaSuccess ||
                (e = lin(z, z, 1.0, df, c_f, hdp, c_p, nullptr, 0, 0.0, st)) != cudaSuccess ||
                (e = H(lp, z, vnew, st)) != cudaSuccess ||
                (e = lin(lap, vnew, 1.0 / a, z, -1.0 / a, nullptr, 0, nullptr, 0, 0.0, st)) != cudaSuccess)
                return fail_f(MOLT_ERR_CUDA, std::string("sixth-order iteration: ") + cudaGetErrorString(e));
            res = read_max(vnew, v, st, &e);
            if (e != cudaSuccess) return fail_f(MOLT_ERR_CUDA, std::string("residual: ") + cudaGetErrorString(e));
            std::swap(v, vnew);
            if (!std::isfinite(res)) break;
            double ulp = 0.0;
            tol_used = p.tol;
            if (fp32) {
                // 2 ulp of max|v| (against the zero field): the FP32 rounding floor of the iterate
                const double vmax = read_max(v, zero, st, &e);
                if (e != cudaSuccess) return fail_f(MOLT_ERR_CUDA, std::string("residual: ") + cudaGetErrorString(e));
                ulp = std::ldexp(1.0, -24) * vmax;
                tol_used = std::max(p.tol, 2.0 * ulp);
            }
            if (res < tol_used) {
                converged = true;
                break;
            }
            if (res < best) {
                best = res;
                stall = 0;
            } else if (fp32 && res < 64.0 * ulp && ++stall >= 6) {
                converged = true;
                tol_used = res;
                break;
            }
        }
        have_lap = true;
        if ((e = lin(u, v, 1.0, nullptr, 0, nullptr, 0, nullptr, 0, -1.0, st)) != cudaSuccess)
            return fail_f(MOLT_ERR_CUDA, std::string("sixth-order store: ") + cudaGetErrorString(e));
        const int it = converged ? k : std::min(k, p.max_iter);
        if (info) {
            info->status = converged ? MOLT_OK : MOLT_ERR_NOT_CONVERGED;
            info->stages = 1;
            info->iters[0] = it;
            info->total_iters = it;
            info->residual = res;
            info->tol_used = tol_used;
        }
        if (!converged)
            molt::set_abi_error(std::isfinite(res) ? "the sixth-order stage reached max_iter before the fixed-point tolerance"
                                                   : "the sixth-order iteration diverged (non-finite residual)");
        return converged ? MOLT_OK : MOLT_ERR_NOT_CONVERGED;
    }
};

}  // namespace

extern "C" {

molt_status molt_fch1d_create(molt_fch1d** out, int nx, int lines, double L, molt_bc bc, double eta,
                              const molt_params* p) {
    if (!out || !p) return fail_f(MOLT_ERR_ARG, "null output handle or parameters");
    *out = nullptr;
    if (bc != MOLT_BC_PERIODIC && bc != MOLT_BC_NEUMANN)
        return fail_f(MOLT_ERR_UNSUPPORTED, "sixth-order steps support periodic and Neumann lines");
    if (p->precision != MOLT_FP32 && p->precision != MOLT_FP64)
        return fail_f(MOLT_ERR_ARG, "precision must be MOLT_FP32 or MOLT_FP64");
    if (p->quad_order != 2 && p->quad_order != 4 && p->quad_order != 6)
        return fail_f(MOLT_ERR_ARG, "quad_order must be 2, 4 or 6");
    if (!(p->eps > 0.0) || !std::isfinite(p->eps) || !(p->tol > 0.0) || p->max_iter < 1)
        return fail_f(MOLT_ERR_ARG, "eps and tol must be positive, max_iter >= 1");
    if (!std::isfinite(eta)) return fail_f(MOLT_ERR_ARG, "eta must be finite");
    const bool f32 = p->precision == MOLT_FP32;
    const int maxn = f32 ? molt::max_row_length<float>(1) : molt::max_row_length<double>(1);
    if (nx < p->quad_order + 2 || nx > maxn)
        return fail_f(MOLT_ERR_ARG, "nx must lie in [M + 2, " + std::to_string(maxn) + "]");
    if (lines < 1 || lines > (1 << 24)) return fail_f(MOLT_ERR_ARG, "lines must lie in [1, 2^24]");
    if (!(L > 0.0) || !std::isfinite(L)) return fail_f(MOLT_ERR_ARG, "L must be finite and > 0");
    molt_fch1d* s = nullptr;
    bool ok = false;
    if (f32) {
        auto* q = new (std::nothrow) Fch1d<float>();
        if (q) {
            q->nx = nx, q->lines = lines, q->bc = bc, q->L = L, q->eta = eta, q->p = *p;
            q->n = static_cast<size_t>(nx) * lines;
            ok = q->init();
        }
        s = q;
    } else {
        auto* q = new (std::nothrow) Fch1d<double>();
        if (q) {
            q->nx = nx, q->lines = lines, q->bc = bc, q->L = L, q->eta = eta, q->p = *p;
            q->n = static_cast<size_t>(nx) * lines;
            ok = q->init();
        }
        s = q;
    }
    if (!s) return fail_f(MOLT_ERR_OOM, "host allocation failed");
    if (!ok) {
        delete s;
        return fail_f(MOLT_ERR_OOM, "sixth-order device workspace allocation failed");
    }
    *out = s;
    return MOLT_OK;
}

molt_status molt_fch1d_destroy(molt_fch1d* s) {
    delete s;
    return MOLT_OK;
}

long long molt_fch1d_launches(const molt_fch1d* s) { return s ? s->launches : 0; }

molt_status molt_fch1d_step(molt_fch1d* s, void* u, double dt, void* stream, molt_step_info* info) {
    if (info) std::memset(info, 0, sizeof(*info));
    if (!s || !u) return fail_f(MOLT_ERR_ARG, "null solver or field");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail_f(MOLT_ERR_ARG, "dt must be finite and > 0");
    return s->step(u, dt, static_cast<cudaStream_t>(stream), info);
}

}  // extern "C"
