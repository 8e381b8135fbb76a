// Internal declarations shared by the host driver and the sweep kernels.
//
// A "line" is one row (x-sweep) or one column (y-sweep) of a row-major [ny][nx] field.
// Positions along a line are 0..n-1.  Periodic lines have N = n intervals (position n is
// position 0); Neumann / Dirichlet lines have N = n - 1 intervals and both walls as nodes.
#pragma once

#include <cstddef>
#include <cstdint>

namespace molt {

enum Bc { BC_PERIODIC = 0, BC_NEUMANN = 1, BC_DIRICHLET = 2 };

constexpr int kMaxM = 6;           // largest quadrature order
constexpr int kColTileRows = 128;  // rows per column tile of the column sweep kernels
constexpr int kMaxStencil = kMaxM + 1;
constexpr int kMaxWall = kMaxM / 2;

// Everything one application of H_c along one axis needs (Sec. 3.2), precomputed on the
// host in FP64 and passed by value to the kernels.
template <typename T>
struct LineParams {
    int n;          // stored nodes per line
    int N;          // intervals
    int M;          // quadrature order (the kernel is also instantiated on it)
    int bc;         // Bc
    T d;            // e^{-nu}, nu = h / sqrt(c)
    T nu;           // nu in the kernel precision (powers d^k = exp(-nu k))
    // Interior stencil, offsets -M/2..M/2: J^L_j = sum wl[o] v_{j+o-M/2}, J^R_j likewise with wr.
    T wl[kMaxStencil];
    T wr[kMaxStencil];
    // Wall stencils of non-periodic lines (Sec. 3.2 reading: shifted inward, same cell).
    // wlA[j-1]: J^L_j, j = 1..M/2-1, on nodes 0..M.   wrA[j]: J^R_j, j = 0..M/2-1, on nodes 0..M.
    // wlB[j-jb]: J^L_j, j = jb..N with jb = N-M/2+1, on nodes N-M..N.
    // wrB[j-jb]: J^R_j, j = jb..N-1, on nodes N-M..N.
    T wlA[kMaxWall][kMaxStencil];
    T wrA[kMaxWall][kMaxStencil];
    T wlB[kMaxWall][kMaxStencil];
    T wrB[kMaxWall][kMaxStencil];
    // Boundary correction in FP64.  Non-periodic: B_a = bAA I_0 + bAB I_N, B_b = bBA I_0 + bBB I_N
    // with I_0 = I^R_0, I_N = I^L_N.  Periodic: carries X = total / (1 - mu) = total * inv1mmu.
    double bAA, bAB, bBA, bBB;
    double inv1mmu;
};

// Host: build the parameters of H_c on a line of n nodes with spacing h.
// Returns false (and a message) on invalid input.
bool build_line_params(double c, double h, int n, int M, int bc, LineParams<double>* out,
                       const char** err);
template <typename T>
LineParams<T> cast_line_params(const LineParams<double>& p);

// Host: record the message molt_last_error(NULL) returns (entry points without a solver).
void set_abi_error(const char* message);

// Host: count one column kernel launched with TMA tile loads (molt_column_tma_launches).
void count_tma_launch();

// Host: coefficients of the stage equation v - tau F(v) = r (Sec. 2.2 factorization when
// tau >= eps^2, Sec. 2.3 completed square otherwise): the two Helmholtz parameters (inner = the
// larger), beta = tau / c_in and lambda = 2 - (c1 + c2) / tau of the lagged term G.
struct StageParams {
    bool factor;
    double c_in, c_out, beta, lam;
};
StageParams stage_params(double tau, double eps);

// Host: node spacing of a line of n stored nodes over a length L (periodic: L / n).
double grid_h(int n, double L, int bc);

// Host: local quadrature weights of Sec. 3.2 for one stencil (factor 1/2 included).
bool quadrature_weights(double nu, int M, const int* offsets, int side, double* w);

// Scratch for the column (y) sweeps: per (field, tile, column) aggregates and carries.
template <typename T>
struct ColScratch {
    T* aggL;    // [NF][tiles][nlines]
    T* aggR;
    T* carL;
    T* carR;
    int tiles;
    int capacity_lines;   // nlines the buffers were sized for
    int capacity_fields;
    unsigned* status = nullptr;   // device word: bits set by kernels whose bounded waits ran out
};

}  // namespace molt

// ------------------------------------------------------------------------------------------
// Kernel launch layer (implemented per precision in kernels_f32.cu / kernels_f64.cu).
// ------------------------------------------------------------------------------------------
#include <cuda_runtime_api.h>

#include <vector>

namespace molt {

// Which fused prologue/epilogue a sweep runs (see sweep_common.cuh for the formulas).
enum OpKind { OP_COPY = 0, OP_P1, OP_P2, OP_P3, OP_P4, OP_1A, OP_1B, OP_V1, OP_V2, OP_V1A, OP_C3 };

template <typename T>
struct OpArgs {
    const T* in0 = nullptr;
    const T* in1 = nullptr;
    const T* in2 = nullptr;
    const T* in3 = nullptr;
    T* out0 = nullptr;
    T* out1 = nullptr;
    T g2 = 0, g1 = 0, beta = 0, shift = 0;
    T vs = 0;       // vector CH: s = (c1 + c2)/tau
    int comp = 0;   // vector CH: component of the pass
    int variant = 0;   // launch choice (Launch); 0 = the default for the line length and field count
    // Block order over the field, for L2 reuse between consecutive passes (results do not depend
    // on it): rows, bit 0 = lines from the last one up; TMA columns, bit 0 = the aggregate phase
    // from the last tile row up, bit 1 = the same for the final phase.  Other kernels ignore it.
    int order = 0;
};

// Kernel choices of one sweep, picked by the solver's autotuner (the values of molt_launch in
// include/molt.h).  Rows: the pipelined kernel on one block per line or on a two-block cluster per
// line, or the general row kernel; columns: TMA tiles, cp.async tiles or the general kernels.
enum Launch { LAUNCH_DEFAULT = 0, LAUNCH_ROWS_ONE_BLOCK = 1, LAUNCH_ROWS_CLUSTER2 = 2, LAUNCH_ROWS_GENERAL = 3,
              LAUNCH_COLS_TMA = 4, LAUNCH_COLS_CP_ASYNC = 5, LAUNCH_COLS_GENERAL = 6, LAUNCH_ROWS_TENSOR_CORE = 7 };

// Dirichlet grids: set the wall nodes of a [ny][nx] field (ny = 1: a line) to `value`, the stored
// form of v = 0 (the boundary data every Dirichlet line inverse holds exactly).
template <typename T>
cudaError_t set_walls(T* w, int nx, int ny, double value, cudaStream_t st, long long* launches);

// Fill n values with a hash of (seed, index) mapped uniformly to [lo, hi) (autotuner test data).
template <typename T>
cudaError_t fill_pattern(T* p, long long n, unsigned seed, double lo, double hi, cudaStream_t st);

// Optional per-kernel event timing (diagnostic; off unless a solver enables it).
// Slots: rows kernel of op k = k; column aggregate kernel = 8 + k; column carry = 16;
// column final kernel = 17 + k.
constexpr int kProfSlots = 32;
struct Prof {
    bool on = false;
    struct Mark { int slot; int a, b; };   // indices into the event pool
    std::vector<Mark> marks;
    std::vector<cudaEvent_t> pool;
    size_t used = 0;
    // record an event before (begin) / after (end) one kernel launch on `st`
    bool begin(int slot, cudaStream_t st);
    void end(cudaStream_t st);
    // wait for the recorded events, add elapsed ms and launch counts per slot, forget the marks
    cudaError_t collect(double* ms, long long* count);
    void release();
};

// Fields are [ny][nx]; axis 0 sweeps the ny rows (lines of nx), axis 1 the nx columns.
template <typename T>
cudaError_t sweep(int axis, const LineParams<T>& lp, int kind, const OpArgs<T>& a, int nx, int ny,
                  ColScratch<T>* cs, unsigned long long* red, cudaStream_t st, long long* launches,
                  Prof* prof = nullptr);

// Largest line length the row kernel supports for a field count (shared-memory bound).
template <typename T>
int max_row_length(int nf);

// out = c0 x0 + c1 x1 + c2 x2 + c3 x3 + c4 (null inputs are skipped), n elements.
template <typename T>
cudaError_t lincomb(T* out, long long n, const T* x0, double c0, const T* x1, double c1, const T* x2,
                    double c2, const T* x3, double c3, double c4, cudaStream_t st, long long* launches);

// Device-side state of one fixed-point stage loop (graph execution mode).
struct LoopState {
    int k;            // iterations done
    int stall;        // iterations without a new residual minimum
    int done;         // loop finished
    int converged;    // finished by the tolerance (or at FP32 precision)
    double best;      // smallest residual so far
    double res;       // last residual max |w_new - w|
    double tol_used;  // tolerance applied at the last check
};

// Reset the loop state and the residual slots (one thread).
cudaError_t loop_init(LoopState* ls, unsigned long long* red, cudaStream_t st);
// Read the residual slots, apply the stopping rule of the host loop (tolerance, FP32 floor of
// 2 ulp of max|w|, stall at the FP32 noise floor, iteration cap), clear the slots and set the
// conditional of the enclosing WHILE node: 1 = iterate again, 0 = stop.
cudaError_t loop_check(cudaGraphConditionalHandle h, LoopState* ls, unsigned long long* red, double tol,
                       int max_iter, int fp32, cudaStream_t st);

// y[j][i] += sum_k a[k][j] b[k][i] (k < terms <= 4), the sum in FP64, for a [ny][nx] field.
struct Separable {
    const double* a[4];
    const double* b[4];
    int terms;
};
template <typename T>
cudaError_t add_separable(T* y, int nx, int ny, const Separable& s, cudaStream_t st, long long* launches);

// Dirichlet grids store w = v - 1: the fixed offset C of a stage's Y as a sum of products of FP64
// line profiles (solver.cpp), from the line parameters of the stage's inner / outer inverses along
// x and y (lp[0..3] = ix, ox, iy, oy; 1D: lp[0..1]) and beta g0 = beta (lambda - 2).
constexpr int kOffsetProfiles = 16;
cudaError_t dirichlet_offset(const LineParams<double> lp[4], int dim, double bg, double* prof, int L, Separable* out,
                             cudaStream_t st, long long* launches);

// Tensor-core row sweep of H_c on periodic FP32 lines (rows_tc.cu): workspace bytes, the line
// lengths and line counts it takes, the one-time operand build for a line inverse, the sweep.
size_t rows_tc_workspace_bytes();
bool rows_tc_supported(int n, int nlines, int M);
cudaError_t rows_tc_prepare(const LineParams<double>& lp, void* workspace, cudaStream_t st);
cudaError_t rows_tc(const LineParams<double>& lp, const void* workspace, const float* in, float* out, int nlines,
                    unsigned* status, cudaStream_t st);

// out = x (x (x + a2) + a1), n elements (the pointwise cubic f of Eq. CahnHilliard_v).
template <typename T>
cudaError_t cubic(T* out, long long n, const T* x, double a2, double a1, cudaStream_t st, long long* launches);

// FP64 energy / mass partial sums: per-block partials into `partials` (>= reduce_blocks()),
// then a single-block fixed-order sum into `result`.
template <typename T>
cudaError_t energy_mass(const T* u, int nx, int ny, int bc, double hx, double hy, double eps,
                        int which, double* partials, double* result, cudaStream_t st,
                        long long* launches);
int reduce_blocks();

// max |a - b| over n values as FP64 bits in *out (device word; zeroed here), for step-size control.
template <typename T>
cudaError_t max_abs_diff(const T* a, const T* b, long long n, unsigned long long* out, cudaStream_t st);

// Sixth-order model, pointwise: f_out = f(v) = v^3 - 3v^2 + 2v and
// p_out = -eps2 f'(v) lap + f f'(v) - eta_eps2 f(v), n elements.
template <typename T>
cudaError_t fch_pointwise(long long n, const T* v, const T* lap, double eps2, double eta_eps2, T* f_out, T* p_out,
                          cudaStream_t st, long long* launches);

}  // namespace molt
