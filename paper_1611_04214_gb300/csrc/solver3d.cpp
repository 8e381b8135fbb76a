// Three-dimensional split stage solve, FP32 (the extension of the 2D splitting that Sec. 5
// remarks on; the paper does not write it out).
//
// With L_a = I - c d_aa on each axis, I - c Lap = L_x L_y L_z - P and
// P = c^2 (dxx dyy + dxx dzz + dyy dzz) - c^3 dxx dyy dzz.  With H_a = L_a^{-1}, D_a = I - H_a and
// M^{-1} = H_x H_y H_z this gives M^{-1} P = X = D_x D_y + D_x D_z + D_y D_z - 2 D_x D_y D_z, i.e.
// I - c Lap = M (I - X).  In 2D the same steps give X = D_x D_y, and the 2D iteration of
// Sec. 5.1 carries over with X in its place:
//   v^{k+1} = Y + M_o^{-1}[beta (M_i^{-1} G - G + X_i G)] + (X_o + X_i - X_o X_i) v^k.
// Written with the pair and triple products of the line inverses,
//   Q f  = (H_x H_y + H_y H_z + H_x H_z - 2 H_x H_y H_z) f   (= (I - X) f),
//   A f  = (3 H_x H_y H_z - H_x H_y - H_y H_z - H_x H_z) f   (= (M^{-1} - I + X) f),
// and in the stored variable w = v - 1 = u (periodic and Neumann lines reproduce constants, so
// the constant lam - 2 of G drops out, as in 2D), one iteration is
//   w^{k+1} = Y + w^k + H_ox H_oy H_oz [beta A_i g] - Q_o [Q_i w^k],   g = w^3 + (lam - 3) w,
// with Y = M_o^{-1} M_i^{-1} r.  Every product is a sequence of single line sweeps: x lines are
// the rows of the [nz * ny][nx] view, z lines the columns of the [nz][ny * nx] view, and the y
// lines of each z slab are the columns of one instance of an internal batch of nz slabs
// (molt_batch_helmholtz_apply), so every sweep is one launch sequence over the whole field.
// By linearity of H_x, Q and A need one x sweep each after combining their y and z products, and
// that combination is fused into the x sweep's prologue and epilogue: 15 line sweeps and one
// linear combination per iteration, the other passes not fused.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <initializer_list>
#include <string>
#include <vector>

#include "../../include/molt.h"
#include "molt_internal.h"

struct molt_solver3d {
    int nx = 0, ny = 0, nz = 0;
    double Lx = 0, Ly = 0, Lz = 0;
    int bc = 0;
    molt_params p{};
    size_t n = 0;
    std::vector<void*> allocs;
    float *w = nullptr, *wn = nullptr, *r = nullptr, *uprev = nullptr, *Y = nullptr, *g = nullptr,
          *zero = nullptr;
    float *hz = nullptr, *hy = nullptr, *hyz = nullptr;   // H_z f, H_y f, H_y H_z f of the current product
    float *tb = nullptr, *qi = nullptr, *qo = nullptr, *hb = nullptr;   // the iteration's terms
    molt::ColScratch<float> cs{};
    unsigned long long* red = nullptr;
    unsigned long long* red_host = nullptr;
    unsigned* status = nullptr;
    unsigned* status_host = nullptr;
    molt_batch* slabs = nullptr;          // nz instances of ny x nx: the y sweeps
    std::vector<double> cbuf;             // nz copies of c for the batched y sweep
    bool have_prev = false;
    double dt_prev = 0.0;
    long long launches = 0;

    ~molt_solver3d() {
        if (slabs) molt_batch_destroy(slabs);
        for (void* q : allocs) cudaFree(q);
        if (red_host) cudaFreeHost(red_host);
        if (status_host) cudaFreeHost(status_host);
    }

    bool alloc(float** q, size_t count) {
        void* v = nullptr;
        if (cudaMalloc(&v, count * sizeof(float)) != cudaSuccess) return false;
        allocs.push_back(v);
        *q = static_cast<float*>(v);
        return true;
    }

    double h(int axis) const {
        const int m = axis == 0 ? nx : axis == 1 ? ny : nz;
        const double L = axis == 0 ? Lx : axis == 1 ? Ly : Lz;
        return molt::grid_h(m, L, bc);
    }
};

namespace {

molt_status fail3(molt_status s, const std::string& m) {
    molt::set_abi_error(m.c_str());
    return s;
}

// One H_c sweep along axis 0 (x), 1 (y) or 2 (z).
cudaError_t sweep3(molt_solver3d* s, int axis, double c, const float* in, float* out, cudaStream_t st) {
    if (axis == 1) {
        std::fill(s->cbuf.begin(), s->cbuf.end(), c);
        const molt_status ms = molt_batch_helmholtz_apply(s->slabs, 1, s->cbuf.data(), in, out, st);
        s->launches += 3;
        return ms == MOLT_OK ? cudaSuccess : cudaErrorUnknown;
    }
    const int m = axis == 0 ? s->nx : s->nz;
    molt::LineParams<double> lpd;
    const char* err = nullptr;
    if (!molt::build_line_params(c, s->h(axis), m, s->p.quad_order, s->bc, &lpd, &err)) return cudaErrorInvalidValue;
    const molt::LineParams<float> lp = molt::cast_line_params<float>(lpd);
    molt::OpArgs<float> a;
    a.in0 = in;
    a.out0 = out;
    if (axis == 0)   // rows of the [nz * ny][nx] view
        return molt::sweep<float>(0, lp, molt::OP_COPY, a, s->nx, s->ny * s->nz, &s->cs, s->red, st, &s->launches);
    // columns of the [nz][ny * nx] view
    return molt::sweep<float>(1, lp, molt::OP_COPY, a, s->nx * s->ny, s->nz, &s->cs, s->red, st, &s->launches);
}

// The y and z products of f at one c: hz = H_z f, hy = H_y f, hyz = H_y H_z f.  The x
// sweeps come after a combination: by linearity of H_x,
//   Q f = H_x H_y f + H_x H_z f + H_y H_z f - 2 H_x H_y H_z f = H_x (H_y f + H_z f - 2 H_y H_z f) + H_y H_z f,
//   A f = 3 H_x H_y H_z f - H_x H_y f - H_x H_z f - H_y H_z f = H_x (3 H_y H_z f - H_y f - H_z f) - H_y H_z f,
// so each takes one x sweep instead of three.
cudaError_t yz_products(molt_solver3d* s, double c, const float* f, cudaStream_t st) {
    cudaError_t e;
    if ((e = sweep3(s, 2, c, f, s->hz, st)) != cudaSuccess || (e = sweep3(s, 1, c, f, s->hy, st)) != cudaSuccess)
        return e;
    return sweep3(s, 1, c, s->hz, s->hyz, st);
}

// out = scale (H_x (a (H_y f + H_z f) + b H_y H_z f) + sign H_y H_z f): Q f for (a, b, sign) =
// (1, -2, +1), A f for (-1, 3, -1).  The combination and the x sweep are one fused row pass
// (OpComb3).  Uses hz, hy, hyz.
cudaError_t q_or_a(molt_solver3d* s, double c, const float* f, double a, double b, double sign, double scale,
                   float* out, cudaStream_t st) {
    cudaError_t e;
    if ((e = yz_products(s, c, f, st)) != cudaSuccess) return e;
    molt::LineParams<double> lpd;
    const char* err = nullptr;
    if (!molt::build_line_params(c, s->h(0), s->nx, s->p.quad_order, s->bc, &lpd, &err)) return cudaErrorInvalidValue;
    const molt::LineParams<float> lp = molt::cast_line_params<float>(lpd);
    molt::OpArgs<float> oa;
    oa.in0 = s->hy;
    oa.in1 = s->hz;
    oa.in2 = s->hyz;
    oa.out0 = out;
    oa.g2 = static_cast<float>(scale * a);
    oa.g1 = static_cast<float>(scale * b);
    oa.beta = static_cast<float>(scale * sign);
    return molt::sweep<float>(0, lp, molt::OP_C3, oa, s->nx, s->ny * s->nz, &s->cs, s->red, st, &s->launches);
}

// out = H_x H_y H_z f (tmp: two scratch fields).
cudaError_t triple(molt_solver3d* s, double c, const float* f, float* out, float* tmp0, float* tmp1,
                   cudaStream_t st) {
    cudaError_t e;
    if ((e = sweep3(s, 2, c, f, tmp0, st)) != cudaSuccess || (e = sweep3(s, 1, c, tmp0, tmp1, st)) != cudaSuccess)
        return e;
    return sweep3(s, 0, c, tmp1, out, st);
}

}  // namespace

namespace {

// One fixed-point iteration: wn = Y + w + H_ox H_oy H_oz [beta A_i g] - Q_o [Q_i w].
cudaError_t iteration3(molt_solver3d* s, const molt::StageParams& sp, cudaStream_t st) {
    const long long n = static_cast<long long>(s->n);
    float* tb = s->tb;   // beta A_i g
    float* qi = s->qi;   // Q_i w
    float* qo = s->qo;   // Q_o Q_i w
    float* hb = s->hb;   // H_ox H_oy H_oz (beta A_i g)
    cudaError_t e;
    // g = w^3 + (lam - 3) w
    if ((e = molt::cubic<float>(s->g, n, s->w, 0.0, sp.lam - 3.0, st, &s->launches)) != cudaSuccess ||
        (e = q_or_a(s, sp.c_in, s->g, -1.0, 3.0, -1.0, sp.beta, tb, st)) != cudaSuccess ||
        (e = q_or_a(s, sp.c_in, s->w, 1.0, -2.0, 1.0, 1.0, qi, st)) != cudaSuccess ||
        (e = triple(s, sp.c_out, tb, hb, s->hz, s->hy, st)) != cudaSuccess ||
        (e = q_or_a(s, sp.c_out, qi, 1.0, -2.0, 1.0, 1.0, qo, st)) != cudaSuccess)
        return e;
    return molt::lincomb<float>(s->wn, n, s->Y, 1.0, s->w, 1.0, hb, 1.0, qo, -1.0, 0.0, st, &s->launches);
}

double read_max(molt_solver3d* s, const float* a, const float* b, cudaStream_t st, cudaError_t* e) {
    double v = 0.0;
    if ((*e = molt::max_abs_diff<float>(a, b, static_cast<long long>(s->n), s->red, st)) != cudaSuccess ||
        (*e = cudaMemcpyAsync(s->red_host, s->red, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st)) !=
            cudaSuccess ||
        (*e = cudaStreamSynchronize(st)) != cudaSuccess)
        return 0.0;
    std::memcpy(&v, s->red_host, sizeof(double));
    s->launches += 1;
    return v;
}

// Stage v - tau F(v) = r (w-form: r and w hold u), first guess in s->w.  The stopping rule is the
// single-grid solver's: ||w^{k+1} - w^k||_inf < tol (Sec. 4.4), the tolerance floored at 2 ulp
// of max|w| in FP32, and an iteration that has not set a new residual minimum for 6 iterations
// while below 64 ulp stops at the FP32 rounding floor.
molt_status stage3(molt_solver3d* s, double tau, cudaStream_t st, int* iters, double* res_out, double* tol_out) {
    const molt::StageParams sp = molt::stage_params(tau, s->p.eps);
    cudaError_t e;
    if ((e = cudaMemsetAsync(s->status, 0, sizeof(unsigned), st)) != cudaSuccess ||
        (e = triple(s, sp.c_in, s->r, s->tb, s->hz, s->hy, st)) != cudaSuccess ||
        (e = triple(s, sp.c_out, s->tb, s->Y, s->hz, s->hy, st)) != cudaSuccess)
        return fail3(MOLT_ERR_CUDA, std::string("3D rhs inverse: ") + cudaGetErrorString(e));
    double res = INFINITY, best = INFINITY, tol_used = s->p.tol;
    int k = 0, stall = 0;
    bool converged = false;
    for (k = 1; k <= s->p.max_iter; ++k) {
        if ((e = iteration3(s, sp, st)) != cudaSuccess)
            return fail3(MOLT_ERR_CUDA, std::string("3D iteration: ") + cudaGetErrorString(e));
        res = read_max(s, s->wn, s->w, st, &e);
        const double wmax = e == cudaSuccess ? read_max(s, s->wn, s->zero, st, &e) : 0.0;
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(s->status_host, s->status, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return fail3(MOLT_ERR_CUDA, std::string("3D residual: ") + cudaGetErrorString(e));
        if (*s->status_host)
            return fail3(MOLT_ERR_CUDA, "a column kernel's bounded wait for a tile copy ran out; the field is incomplete");
        std::swap(s->w, s->wn);
        if (!std::isfinite(res)) break;
        const double ulp = std::ldexp(1.0, -24) * wmax;
        tol_used = std::max(s->p.tol, 2.0 * ulp);
        if (res < tol_used) {
            converged = true;
            break;
        }
        if (res < best) {
            best = res;
            stall = 0;
        } else if (res < 64.0 * ulp && ++stall >= 6) {
            converged = true;
            tol_used = res;
            break;
        }
    }
    *iters = converged ? k : std::min(k, s->p.max_iter);
    *res_out = res;
    *tol_out = tol_used;
    if (!converged)
        molt::set_abi_error(std::isfinite(res) ? "the 3D stage reached max_iter before the fixed-point tolerance"
                                               : "the 3D iteration diverged (non-finite residual)");
    return converged ? MOLT_OK : MOLT_ERR_NOT_CONVERGED;
}

}  // namespace

extern "C" {

molt_status molt_solver3d_create(molt_solver3d** out, int nx, int ny, int nz, double Lx, double Ly, double Lz,
                                 molt_bc bc, const molt_params* p) {
    if (!out || !p) return fail3(MOLT_ERR_ARG, "null output handle or parameters");
    *out = nullptr;
    if (bc != MOLT_BC_PERIODIC && bc != MOLT_BC_NEUMANN)
        return fail3(MOLT_ERR_UNSUPPORTED, "3D steps support periodic and Neumann lines");
    if (p->precision != MOLT_FP32) return fail3(MOLT_ERR_UNSUPPORTED, "3D steps run in FP32");
    if (p->quad_order != 2 && p->quad_order != 4 && p->quad_order != 6)
        return fail3(MOLT_ERR_ARG, "quad_order must be 2, 4 or 6");
    if (!(p->eps > 0.0) || !std::isfinite(p->eps) || !(p->tol > 0.0) || p->max_iter < 1)
        return fail3(MOLT_ERR_ARG, "eps and tol must be positive, max_iter >= 1");
    const int lo = p->quad_order + 2;
    if (nx < lo || ny < lo || nz < lo || nx > 1024 || ny > 1024 || nz > (1 << 20))
        return fail3(MOLT_ERR_ARG, "nx, ny must lie in [M + 2, 1024] and nz in [M + 2, 2^20]");
    if (!(Lx > 0.0) || !(Ly > 0.0) || !(Lz > 0.0) || !std::isfinite(Lx) || !std::isfinite(Ly) || !std::isfinite(Lz))
        return fail3(MOLT_ERR_ARG, "Lx, Ly, Lz must be finite and > 0");
    molt_solver3d* s = new (std::nothrow) molt_solver3d();
    if (!s) return fail3(MOLT_ERR_OOM, "host allocation failed");
    s->nx = nx;
    s->ny = ny;
    s->nz = nz;
    s->Lx = Lx;
    s->Ly = Ly;
    s->Lz = Lz;
    s->bc = bc;
    s->p = *p;
    s->n = static_cast<size_t>(nx) * ny * nz;
    s->cbuf.assign(nz, 0.0);
    bool ok = s->alloc(&s->w, s->n) && s->alloc(&s->wn, s->n) && s->alloc(&s->r, s->n) && s->alloc(&s->uprev, s->n) &&
              s->alloc(&s->Y, s->n) && s->alloc(&s->g, s->n) && s->alloc(&s->zero, s->n);
    for (float** q : {&s->hz, &s->hy, &s->hyz, &s->tb, &s->qi, &s->qo, &s->hb}) ok = ok && s->alloc(q, s->n);
    // column scratch of the z sweeps: nx * ny columns of nz nodes
    const int lines = nx * ny, tiles = (nz + molt::kColTileRows - 1) / molt::kColTileRows;
    const size_t sc = static_cast<size_t>(2) * tiles * lines;
    s->cs.tiles = tiles;
    s->cs.capacity_lines = lines;
    s->cs.capacity_fields = 2;
    ok = ok && s->alloc(&s->cs.aggL, sc) && s->alloc(&s->cs.aggR, sc) && s->alloc(&s->cs.carL, sc) &&
         s->alloc(&s->cs.carR, sc);
    void* q = nullptr;
    if (ok && cudaMalloc(&q, 2 * sizeof(unsigned long long)) == cudaSuccess) {
        s->allocs.push_back(q);
        s->red = static_cast<unsigned long long*>(q);
    } else {
        ok = false;
    }
    if (ok && cudaMalloc(&q, sizeof(unsigned)) == cudaSuccess) {
        s->allocs.push_back(q);
        s->status = static_cast<unsigned*>(q);
        s->cs.status = s->status;
    } else {
        ok = false;
    }
    ok = ok && cudaMemset(s->zero, 0, s->n * sizeof(float)) == cudaSuccess &&
         cudaMemset(s->status, 0, sizeof(unsigned)) == cudaSuccess &&
         cudaMallocHost(&s->red_host, 2 * sizeof(unsigned long long)) == cudaSuccess &&
         cudaMallocHost(&s->status_host, sizeof(unsigned)) == cudaSuccess;
    if (!ok) {
        delete s;
        return fail3(MOLT_ERR_OOM, "3D device workspace allocation failed");
    }
    *s->status_host = 0;
    // the y lines: nz instances of ny x nx, back to back = the [nz][ny][nx] layout
    std::vector<molt_instance> inst(nz, molt_instance{nx, ny, Lx, Ly, p->eps});
    const molt_status bs = molt_batch_create(&s->slabs, nz, inst.data(), bc, p->quad_order, p->tol, p->max_iter);
    if (bs != MOLT_OK) {
        s->slabs = nullptr;
        delete s;
        return bs;   // its message is already recorded
    }
    *out = s;
    return MOLT_OK;
}

molt_status molt_solver3d_destroy(molt_solver3d* s) {
    delete s;
    return MOLT_OK;
}

long long molt_solver3d_launches(const molt_solver3d* s) { return s ? s->launches : 0; }

molt_status molt_solver3d_apply(molt_solver3d* s, int axis, double c, const float* in, float* out, void* stream) {
    if (!s || !in || !out) return fail3(MOLT_ERR_ARG, "null solver or field");
    if (axis < 0 || axis > 2) return fail3(MOLT_ERR_ARG, "axis must be 0 (x), 1 (y) or 2 (z)");
    if (in == out) return fail3(MOLT_ERR_ARG, "in and out must not alias");
    if (!(c > 0.0) || !std::isfinite(c)) return fail3(MOLT_ERR_ARG, "c must be positive and finite");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(s->status, 0, sizeof(unsigned), st);
    if (e == cudaSuccess) e = sweep3(s, axis, c, in, out, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->status_host, s->status, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail3(MOLT_ERR_CUDA, std::string("3D sweep: ") + cudaGetErrorString(e));
    if (*s->status_host)
        return fail3(MOLT_ERR_CUDA, "a column kernel's bounded wait for a tile copy ran out; the output is incomplete");
    return MOLT_OK;
}

molt_status molt_solver3d_step(molt_solver3d* s, float* u, double dt, molt_scheme scheme, void* stream,
                               molt_step_info* info) {
    if (info) std::memset(info, 0, sizeof(*info));
    if (!s || !u) return fail3(MOLT_ERR_ARG, "null solver or field");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail3(MOLT_ERR_ARG, "dt must be finite and > 0");
    if (scheme != MOLT_BE && scheme != MOLT_BDF2) return fail3(MOLT_ERR_UNSUPPORTED, "3D steps support BE and BDF2");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t bytes = s->n * sizeof(float);
    const long long n = static_cast<long long>(s->n);
    const bool bdf = scheme == MOLT_BDF2 && s->have_prev && s->dt_prev == dt;
    const double tau = bdf ? 2.0 * dt / 3.0 : dt;
    cudaError_t e = cudaMemcpyAsync(s->w, u, bytes, cudaMemcpyDeviceToDevice, st);   // first guess u^n
    if (e == cudaSuccess)
        e = bdf ? molt::lincomb<float>(s->r, n, u, 4.0 / 3.0, s->uprev, -1.0 / 3.0, nullptr, 0.0, nullptr, 0.0, 0.0, st,
                                       &s->launches)
                : cudaMemcpyAsync(s->r, u, bytes, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return fail3(MOLT_ERR_CUDA, std::string("3D step load: ") + cudaGetErrorString(e));
    int it = 0;
    double res = 0.0, tol_used = s->p.tol;
    const molt_status ms = stage3(s, tau, st, &it, &res, &tol_used);
    if (ms != MOLT_OK && ms != MOLT_ERR_NOT_CONVERGED) return ms;
    if ((e = cudaMemcpyAsync(s->uprev, u, bytes, cudaMemcpyDeviceToDevice, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(u, s->w, bytes, cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
        return fail3(MOLT_ERR_CUDA, std::string("3D step store: ") + cudaGetErrorString(e));
    s->have_prev = scheme == MOLT_BDF2;
    s->dt_prev = dt;
    if (info) {
        info->status = ms;
        info->stages = 1;
        info->iters[0] = it;
        info->total_iters = it;
        info->residual = res;
        info->tol_used = tol_used;
    }
    return ms;
}

}  // extern "C"
