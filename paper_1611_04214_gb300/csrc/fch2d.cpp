// The sixth-order (functionalized) Cahn-Hilliard model of the paper's last section on a 2D grid,
// BE steps (Eq. FCH0 / FCH, the cube of Eq. FCH_BE with the PDE's signs), split as in Sec. 5.1.
//
// With a = (dt eps^4)^(1/3), H_x, H_y the line inverses of I - a d_xx, I - a d_yy (Sec. 3),
// M^{-1} = H_x H_y and X = D_x D_y (D = H - I), I - a Lap = M (I - X) and these commute, so the
// lagged BE iteration is v <- M^{-3} R(v) + (1 - (1 - X)^3) v with
// R(v) = v^n + dt Lap g(v) - (3a Lap - 3a^2 Lap^2) v.  Every Lap comes with an M^{-1} through
// K = M^{-1} a Lap = 2 M^{-1} - H_x - H_y, and the iterate is kept as v = M^{-1} W:
//   W <- M^{-2} v^n - 3 M^{-1} K v + (3 + c_eta) K^2 v - c_f K^2 f + c_p M^{-1} K p
//        + (3X - 3X^2 + X^3) W,
//   c_eta = dt eta eps^4 / a^2, c_f = dt eps^2 / a^2, c_p = dt / a,
//   p = -eps^2 f' Lap v + f f' - eta eps^2 f,  Lap v = K W / a (exact for the discrete operators).
// The first step starts from W = v^n; later steps carry W.  By linearity the terms regroup into
// products of H_x, H_y on a few combinations (with A = (3 + c_eta) v - c_f f, B = -3v + c_p p):
//   C = K A + M^{-1} B = M^{-1} (2A + B) - H_x A - H_y A,
//   D = 3W - 3XW + X^2 W = M^{-1} E - H_x E - H_y E + X W,  E = X W - 3W,
//   W_new = M^{-2} v^n + K C + X D = M^{-2} v^n + M^{-1} (2C + D) - H_x (C + D) - H_y (C + D) + D,
// 14 one-field line sweeps per iteration (11 here, 3 for v, Lap v and X W of the new W; rows
// through the row kernels, columns through the column kernels), one pointwise kernel and 11 linear
// combinations over the [ny][nx] field, then the residual read (one stream synchronization per
// iteration).  The stopping rule is the single-grid solver's (FP32: the
// tolerance floored at 2 ulp of max|v| and the stall rule below 64 ulp).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <initializer_list>
#include <string>
#include <vector>

#include "../../include/molt.h"
#include "molt_internal.h"

struct molt_fch2d {
    virtual ~molt_fch2d() = default;
    virtual molt_status step(void* u, double dt, cudaStream_t st, molt_step_info* info) = 0;
    long long launches = 0;
};

namespace {

molt_status fail2(molt_status s, const std::string& m) {
    molt::set_abi_error(m.c_str());
    return s;
}

template <typename T>
struct Fch2d final : molt_fch2d {
    int nx = 0, ny = 0, bc = 0;
    double Lx = 0.0, Ly = 0.0, eta = 0.0;
    molt_params p{};
    size_t n = 0;
    std::vector<void*> allocs;
    // iterate (v = M^{-1} W), start of step, carried Lap v and the lagged remainder X W
    T *v = nullptr, *vnew = nullptr, *W = nullptr, *Wn = nullptr, *vn = nullptr, *m2vn = nullptr, *lap = nullptr;
    T *xw = nullptr;
    // pointwise parts and the regrouped combinations 2A + B, A, C, E, D, 2C + D, C + D
    T *f = nullptr, *pp = nullptr, *s1 = nullptr, *aa = nullptr, *cc = nullptr, *ee = nullptr, *dd = nullptr;
    T *s2 = nullptr, *s3 = nullptr;
    // sweep outputs and combination scratch
    T *hx = nullptr, *hy = nullptr, *hm = nullptr, *t1 = nullptr, *tt = nullptr, *zero = nullptr;
    molt::ColScratch<T> cs{};
    unsigned* status = nullptr;
    unsigned* status_host = nullptr;
    unsigned long long* red = nullptr;
    unsigned long long* red_host = nullptr;
    bool have_w = false;   // W of the last step's iterate is in `W`

    ~Fch2d() override {
        for (void* q : allocs) cudaFree(q);
        if (red_host) cudaFreeHost(red_host);
        if (status_host) cudaFreeHost(status_host);
    }

    template <typename U>
    bool alloc(U** q, size_t count) {
        void* m = nullptr;
        if (cudaMalloc(&m, count * sizeof(U)) != cudaSuccess) return false;
        allocs.push_back(m);
        *q = static_cast<U*>(m);
        return true;
    }

    bool init() {
        for (T** q : {&v, &vnew, &W, &Wn, &vn, &m2vn, &lap, &xw, &f, &pp, &s1, &aa, &cc, &ee, &dd, &s2, &s3, &hx,
                      &hy, &hm, &t1, &tt, &zero})
            if (!alloc(q, n)) return false;
        // column scan scratch of the y sweeps: nx columns of ny nodes in tiles of kColTileRows rows
        const int tiles = (ny + molt::kColTileRows - 1) / molt::kColTileRows;
        const size_t sc = static_cast<size_t>(2) * tiles * nx;
        cs.tiles = tiles;
        cs.capacity_lines = nx;
        cs.capacity_fields = 2;
        if (!alloc(&cs.aggL, sc) || !alloc(&cs.aggR, sc) || !alloc(&cs.carL, sc) || !alloc(&cs.carR, sc) ||
            !alloc(&red, 2) || !alloc(&status, 1))
            return false;
        cs.status = status;
        if (cudaMemset(zero, 0, n * sizeof(T)) != cudaSuccess || cudaMemset(status, 0, sizeof(unsigned)) != cudaSuccess ||
            cudaMallocHost(&red_host, 2 * sizeof(unsigned long long)) != cudaSuccess ||
            cudaMallocHost(&status_host, sizeof(unsigned)) != cudaSuccess)
            return false;
        *status_host = 0;
        return true;
    }

    struct Lines {
        molt::LineParams<T> x, y;
    };

    // one line inverse along x (axis 0: the ny rows) or y (axis 1: the nx columns)
    cudaError_t H(int axis, const Lines& lp, const T* in, T* out, cudaStream_t st) {
        molt::OpArgs<T> a;
        a.in0 = in;
        a.out0 = out;
        return molt::sweep<T>(axis, axis == 0 ? lp.x : lp.y, molt::OP_COPY, a, nx, ny, &cs, red, st, &launches);
    }

    cudaError_t lin(T* out, const T* x0, double c0, const T* x1, double c1, const T* x2, double c2, const T* x3,
                    double c3, cudaStream_t st) {
        return molt::lincomb<T>(out, static_cast<long long>(n), x0, c0, x1, c1, x2, c2, x3, c3, 0.0, st, &launches);
    }

    // hx = H_x g, hy = H_y g, m = M^{-1} g = H_x H_y g
    cudaError_t parts(const Lines& lp, const T* g, T* m, cudaStream_t st) {
        cudaError_t e;
        if ((e = H(0, lp, g, hx, st)) != cudaSuccess || (e = H(1, lp, g, hy, st)) != cudaSuccess) return e;
        return H(0, lp, hy, m, st);
    }

    // v = M^{-1} W, Lap v = K W / a and X W, from the current W
    cudaError_t from_w(const Lines& lp, const T* w, T* vout, double a, cudaStream_t st) {
        cudaError_t e;
        if ((e = parts(lp, w, vout, st)) != cudaSuccess ||
            (e = lin(lap, vout, 2.0 / a, hx, -1.0 / a, hy, -1.0 / a, nullptr, 0.0, st)) != cudaSuccess)
            return e;
        return lin(xw, vout, 1.0, hx, -1.0, hy, -1.0, w, 1.0, st);
    }

    // max |a - b| (FP64 bits through the reduction word) and the column kernels' wait status
    double read_max(const T* a, const T* b, cudaStream_t st, cudaError_t* e) {
        double r = 0.0;
        if ((*e = molt::max_abs_diff<T>(a, b, static_cast<long long>(n), red, st)) != cudaSuccess ||
            (*e = cudaMemcpyAsync(red_host, red, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st)) !=
                cudaSuccess ||
            (*e = cudaMemcpyAsync(status_host, status, sizeof(unsigned), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
            (*e = cudaStreamSynchronize(st)) != cudaSuccess)
            return 0.0;
        std::memcpy(&r, red_host, sizeof(double));
        launches += 1;
        return r;
    }

    bool line_params(double a, Lines* lp, std::string* err) {
        molt::LineParams<double> px, py;
        const char* m = nullptr;
        if (!molt::build_line_params(a, molt::grid_h(nx, Lx, bc), nx, p.quad_order, bc, &px, &m) ||
            !molt::build_line_params(a, molt::grid_h(ny, Ly, bc), ny, p.quad_order, bc, &py, &m)) {
            *err = m ? m : "bad line parameters";
            return false;
        }
        lp->x = molt::cast_line_params<T>(px);
        lp->y = molt::cast_line_params<T>(py);
        return true;
    }

    molt_status step(void* uv, double dt, cudaStream_t st, molt_step_info* info) override;
};

}  // namespace

namespace {

template <typename T>
molt_status Fch2d<T>::step(void* uv, double dt, cudaStream_t st, molt_step_info* info) {
    T* u = static_cast<T*>(uv);
    const double eps = p.eps;
    const double a = std::cbrt(dt * eps * eps * eps * eps);
    const double c_eta = dt * eta * std::pow(eps, 4) / (a * a), c_f = dt * eps * eps / (a * a), c_p = dt / a;
    Lines lp;
    std::string perr;
    if (!line_params(a, &lp, &perr)) return fail2(MOLT_ERR_ARG, perr);
    cudaError_t e;
    // v^n = u + 1 and M^{-2} v^n; W = v^n for initial data, else the carried W; v, Lap v, X W
    if ((e = cudaMemsetAsync(status, 0, sizeof(unsigned), st)) != cudaSuccess ||
        (e = molt::lincomb<T>(vn, static_cast<long long>(n), u, 1.0, nullptr, 0.0, nullptr, 0.0, nullptr, 0.0, 1.0, st,
                              &launches)) != cudaSuccess ||
        (e = H(1, lp, vn, hy, st)) != cudaSuccess || (e = H(0, lp, hy, hm, st)) != cudaSuccess ||
        (e = H(1, lp, hm, hy, st)) != cudaSuccess || (e = H(0, lp, hy, m2vn, st)) != cudaSuccess ||
        (!have_w && (e = lin(W, vn, 1.0, nullptr, 0.0, nullptr, 0.0, nullptr, 0.0, st)) != cudaSuccess) ||
        (e = from_w(lp, W, v, a, st)) != cudaSuccess)
        return fail2(MOLT_ERR_CUDA, std::string("sixth-order 2D step load: ") + cudaGetErrorString(e));
    double res = INFINITY, best = INFINITY, tol_used = p.tol;
    int k = 0, stall = 0;
    bool converged = false;
    const bool fp32 = sizeof(T) == 4;
    for (k = 1; k <= p.max_iter; ++k) {
        if ((e = molt::fch_pointwise<T>(static_cast<long long>(n), v, lap, eps * eps, eta * eps * eps, f, pp, st,
                                        &launches)) != cudaSuccess ||
            // 2A + B and A
            (e = lin(s1, v, 3.0 + 2.0 * c_eta, f, -2.0 * c_f, pp, c_p, nullptr, 0.0, st)) != cudaSuccess ||
            (e = lin(aa, v, 3.0 + c_eta, f, -c_f, nullptr, 0.0, nullptr, 0.0, st)) != cudaSuccess ||
            // C = M^{-1} (2A + B) - H_x A - H_y A
            (e = H(1, lp, s1, t1, st)) != cudaSuccess || (e = H(0, lp, t1, hm, st)) != cudaSuccess ||
            (e = H(0, lp, aa, hx, st)) != cudaSuccess || (e = H(1, lp, aa, hy, st)) != cudaSuccess ||
            (e = lin(cc, hm, 1.0, hx, -1.0, hy, -1.0, nullptr, 0.0, st)) != cudaSuccess ||
            // E = X W - 3W, D = M^{-1} E - H_x E - H_y E + X W
            (e = lin(ee, W, -3.0, xw, 1.0, nullptr, 0.0, nullptr, 0.0, st)) != cudaSuccess ||
            (e = H(1, lp, ee, t1, st)) != cudaSuccess || (e = H(0, lp, t1, hm, st)) != cudaSuccess ||
            (e = H(0, lp, ee, hx, st)) != cudaSuccess ||
            (e = lin(dd, hm, 1.0, hx, -1.0, t1, -1.0, xw, 1.0, st)) != cudaSuccess ||
            // W_new = M^{-2} v^n + M^{-1} (2C + D) - H_x (C + D) - H_y (C + D) + D
            (e = lin(s2, cc, 2.0, dd, 1.0, nullptr, 0.0, nullptr, 0.0, st)) != cudaSuccess ||
            (e = lin(s3, cc, 1.0, dd, 1.0, nullptr, 0.0, nullptr, 0.0, st)) != cudaSuccess ||
            (e = H(1, lp, s2, t1, st)) != cudaSuccess || (e = H(0, lp, t1, hm, st)) != cudaSuccess ||
            (e = H(0, lp, s3, hx, st)) != cudaSuccess || (e = H(1, lp, s3, hy, st)) != cudaSuccess ||
            (e = lin(tt, hm, 1.0, hx, -1.0, hy, -1.0, dd, 1.0, st)) != cudaSuccess ||
            (e = lin(Wn, tt, 1.0, m2vn, 1.0, nullptr, 0.0, nullptr, 0.0, st)) != cudaSuccess ||
            (e = from_w(lp, Wn, vnew, a, st)) != cudaSuccess)
            return fail2(MOLT_ERR_CUDA, std::string("sixth-order 2D iteration: ") + cudaGetErrorString(e));
        res = read_max(vnew, v, st, &e);
        if (e != cudaSuccess) return fail2(MOLT_ERR_CUDA, std::string("residual: ") + cudaGetErrorString(e));
        if (*status_host)
            return fail2(MOLT_ERR_CUDA, "a column kernel's bounded wait for a tile copy ran out; the field is incomplete");
        std::swap(v, vnew);
        std::swap(W, Wn);
        if (!std::isfinite(res)) break;
        double ulp = 0.0;
        tol_used = p.tol;
        if (fp32) {
            // 2 ulp of max|v| (against the zero field): the FP32 rounding floor of the iterate
            const double vmax = read_max(v, zero, st, &e);
            if (e != cudaSuccess) return fail2(MOLT_ERR_CUDA, std::string("residual: ") + cudaGetErrorString(e));
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
    have_w = true;
    if ((e = molt::lincomb<T>(u, static_cast<long long>(n), v, 1.0, nullptr, 0.0, nullptr, 0.0, nullptr, 0.0, -1.0, st,
                              &launches)) != cudaSuccess)
        return fail2(MOLT_ERR_CUDA, std::string("sixth-order 2D store: ") + cudaGetErrorString(e));
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
        molt::set_abi_error(std::isfinite(res) ? "the sixth-order 2D stage reached max_iter before the fixed-point tolerance"
                                               : "the sixth-order 2D iteration diverged (non-finite residual)");
    return converged ? MOLT_OK : MOLT_ERR_NOT_CONVERGED;
}

template <typename T>
molt_status make(molt_fch2d** out, int nx, int ny, double Lx, double Ly, int bc, double eta, const molt_params* p) {
    auto* s = new (std::nothrow) Fch2d<T>();
    if (!s) return fail2(MOLT_ERR_OOM, "host allocation failed");
    s->nx = nx, s->ny = ny, s->bc = bc, s->Lx = Lx, s->Ly = Ly, s->eta = eta, s->p = *p;
    s->n = static_cast<size_t>(nx) * ny;
    if (!s->init()) {
        delete s;
        return fail2(MOLT_ERR_OOM, "sixth-order 2D device workspace allocation failed");
    }
    *out = s;
    return MOLT_OK;
}

}  // namespace

extern "C" {

molt_status molt_fch2d_create(molt_fch2d** out, int nx, int ny, double Lx, double Ly, molt_bc bc, double eta,
                              const molt_params* p) {
    if (!out || !p) return fail2(MOLT_ERR_ARG, "null output handle or parameters");
    *out = nullptr;
    if (bc != MOLT_BC_PERIODIC && bc != MOLT_BC_NEUMANN)
        return fail2(MOLT_ERR_UNSUPPORTED, "sixth-order 2D steps support periodic and Neumann lines");
    if (p->precision != MOLT_FP32 && p->precision != MOLT_FP64)
        return fail2(MOLT_ERR_ARG, "precision must be MOLT_FP32 or MOLT_FP64");
    if (p->quad_order != 2 && p->quad_order != 4 && p->quad_order != 6)
        return fail2(MOLT_ERR_ARG, "quad_order must be 2, 4 or 6");
    if (!(p->eps > 0.0) || !std::isfinite(p->eps) || !(p->tol > 0.0) || p->max_iter < 1)
        return fail2(MOLT_ERR_ARG, "eps and tol must be positive, max_iter >= 1");
    if (!std::isfinite(eta)) return fail2(MOLT_ERR_ARG, "eta must be finite");
    const bool f32 = p->precision == MOLT_FP32;
    const int maxn = f32 ? molt::max_row_length<float>(1) : molt::max_row_length<double>(1);
    const int lo = p->quad_order + 2;
    if (nx < lo || nx > maxn || ny < lo)
        return fail2(MOLT_ERR_ARG, "nx must lie in [M + 2, " + std::to_string(maxn) + "] and ny >= M + 2");
    if (static_cast<long long>(nx) * ny > (1LL << 31) - 1) return fail2(MOLT_ERR_ARG, "grid too large");
    if (!(Lx > 0.0) || !(Ly > 0.0) || !std::isfinite(Lx) || !std::isfinite(Ly))
        return fail2(MOLT_ERR_ARG, "Lx and Ly must be finite and > 0");
    return f32 ? make<float>(out, nx, ny, Lx, Ly, bc, eta, p) : make<double>(out, nx, ny, Lx, Ly, bc, eta, p);
}

molt_status molt_fch2d_destroy(molt_fch2d* s) {
    delete s;
    return MOLT_OK;
}

long long molt_fch2d_launches(const molt_fch2d* s) { return s ? s->launches : 0; }

molt_status molt_fch2d_step(molt_fch2d* s, void* u, double dt, void* stream, molt_step_info* info) {
    if (info) std::memset(info, 0, sizeof(*info));
    if (!s || !u) return fail2(MOLT_ERR_ARG, "null solver or field");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail2(MOLT_ERR_ARG, "dt must be finite and > 0");
    return s->step(u, dt, static_cast<cudaStream_t>(stream), info);
}

}  // extern "C"
