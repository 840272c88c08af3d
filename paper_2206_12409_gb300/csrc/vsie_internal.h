// Internal declarations of libvsie (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>
#include <complex>

#include "../../include/vsie.h"

namespace vsie {

template <int N> struct int_ {};

// ----------------------------------------------------------------- complex math
template <typename R> struct cx_of;
template <> struct cx_of<float> { using type = float2; };
template <> struct cx_of<double> { using type = double2; };
template <typename R> using cx = typename cx_of<R>::type;

template <typename C> __host__ __device__ __forceinline__ C mk(double re, double im) {
    C c; c.x = re; c.y = im; return c;
}
__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
__host__ __device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
    return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
__host__ __device__ __forceinline__ double2 cmulc(double2 a, double2 b) {
    return make_double2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
// acc += a * b
__host__ __device__ __forceinline__ void cfma(float2& acc, float2 a, float2 b) {
    acc.x = fmaf(a.x, b.x, acc.x); acc.x = fmaf(-a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y); acc.y = fmaf(a.y, b.x, acc.y);
}
__host__ __device__ __forceinline__ void cfma(double2& acc, double2 a, double2 b) {
    acc.x = fma(a.x, b.x, acc.x); acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y); acc.y = fma(a.y, b.x, acc.y);
}
__host__ __device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__host__ __device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__host__ __device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__host__ __device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
template <typename C> __host__ __device__ __forceinline__ C czero() { C c; c.x = 0; c.y = 0; return c; }
template <typename C> __host__ __device__ __forceinline__ C make_neg(C a) { a.x = -a.x; a.y = -a.y; return a; }

// Convert between precisions (device and host).
__host__ __device__ __forceinline__ float2 to_c(float2 a, float2*) { return a; }
__host__ __device__ __forceinline__ double2 to_c(double2 a, double2*) { return a; }
__host__ __device__ __forceinline__ float2 to_c(double2 a, float2*) { return make_float2((float)a.x, (float)a.y); }
__host__ __device__ __forceinline__ double2 to_c(float2 a, double2*) { return make_double2(a.x, a.y); }

// ----------------------------------------------------------------- FFT plans
constexpr int kMaxStages = 16;
constexpr double kEps0 = 8.8541878128e-12;   // F/m (CODATA 2018)
constexpr double kC0 = 299792458.0;          // m/s

// One 1D FFT length: radix sequence (first stage first) and twiddle table
// tw[m] = exp(-2 pi i m / L), m in [0, L), in both precisions.
struct FFTPlan {
    int L = 0;
    int nst = 0;
    int rad[kMaxStages] = {0};
    int ns[kMaxStages] = {0};          // product of the radices before each stage
    uint32_t nsmagic[kMaxStages] = {0};  // floor(2^32 / ns) + 1 (0 when ns == 1)
    int twstep[kMaxStages] = {0};      // L / (ns * rad)
};

// q = x / d for x, d < 2^16 via one multiply-high (exact in that range).
__host__ __device__ inline uint32_t magic_div(uint32_t d) {
    return d <= 1 ? 0u : (uint32_t)((0x100000000ull / d) + 1ull);
}

// radices (16,) 8, 4, 2, 3, 5, 7 with the largest power-of-two radix max_radix;
// false if L is not 7-smooth
bool fft_factor(int L, FFTPlan& plan, int max_radix);
int next_smooth(int n);                    // smallest 7-smooth integer >= n

// ----------------------------------------------------------------- device buffers
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

// Per-precision device data of the operator.
template <typename R>
struct OpData {
    // volume / pFFT
    cx<R>* spec = nullptr;      // 6 octant spectra, scaled by h^3 / (L1 L2 L3)
    cx<R>* tw[3] = {nullptr, nullptr, nullptr};   // twiddles per axis
    cx<R>* dinv = nullptr;      // h^3 / chi per body voxel (0 on vacuum)
    cx<R>* W = nullptr;         // m_n x 3 s^3 projection weights (row per RWG)
    cx<R>* sc_val = nullptr;    // scatter CSR values (active voxel-component rows)
    cx<R>* pre_val = nullptr;   // precorrection CSR (body rows)
    cx<R>* preT_val = nullptr;  // transposed precorrection CSR (RWG rows)
    cx<R>* Znn = nullptr;
    cx<R>* U = nullptr;
    cx<R>* V = nullptr;
    cx<R>* Zff = nullptr;
    cx<R>* G[3][4] = {{nullptr}};   // TT cores; G[c][3] stored transposed (m_f x r3)
    // workspaces
    cx<R>* bufA = nullptr;      // [chunk][3][n3][n2][L1]  (in Ctx::conv_work, shared
    cx<R>* bufB = nullptr;      // [chunk][3][n3][L2][L1]   by both precisions)
    int chunk = 1;              // right-hand sides per launch group of the convolution
    cx<R>* gc = nullptr;        // [p][3][nact] coil contributions on active voxels
    cx<R>* cc = nullptr;        // [p][3][nact] convolution on active voxels
    cx<R>* t1 = nullptr;        // small GEMM intermediates
    cx<R>* t2 = nullptr;
    cx<R>* t3 = nullptr;
    cx<R>* t4 = nullptr;
    cx<R>* splitk = nullptr;    // split-K partial sums
    size_t splitk_elems = 0;
    cx<R>* pc_Zffi = nullptr;   // block preconditioner: Z_ff^-1 (m_f x m_f)
    cx<R>* pc_Znni = nullptr;   // Z_nn^-1 (m_n x m_n)
    cx<R>* pc_bdiag = nullptr;  // inverse body diagonal (n_b)
    int tune[5] = {0, 0, 0, 0, 0};     // chosen FFT pass variants (autotuned)
    float tune_ms[5][16] = {{0}};      // measured time per variant (ms, p = min(chunk, 4))
    bool ready = false;
};

// Per-context profiling: kernel groups, launch counts (always), CUDA-event time
// and algorithmic bytes (when enabled by vsie_profile).
enum ProfGroup { PG_FFTCONV = 0, PG_PFFT = 1, PG_PRECORR = 2, PG_SURF = 3, PG_TT = 4, PG_KRYLOV = 5,
                 PG_PRECOND = 6, PG_FFTCONV64 = 7, PG_N = 8 };
struct Prof {
    bool on = false;
    int group = PG_SURF;                       // group charged by nested launchers
    int64_t launches[PG_N] = {0};
    double alg_bytes[PG_N] = {0};
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev[PG_N];
};

// Hierarchical far-far block (hmatrix.cu): index structures and data, device.
struct HmDev {
    bool on = false;
    int m = 0, nrl = 0, nblk = 0, nlr = 0, nt = 0, ndense = 0, rows_threads = 256;
    int64_t nD = 0, nU = 0, nV = 0;
    int* perm = nullptr;       // cluster position -> RWG index
    int* rl = nullptr;         // leaf row clusters (nrl + 1)
    int4* blk = nullptr;       // (row start, rows, column start, columns) per block
    int* kb = nullptr;         // rank per block, -1 dense
    int64_t* doff = nullptr;   // dense: offset in D; low rank: offset of U
    int64_t* voff = nullptr;   // low rank: offset of V
    int* toff = nullptr;       // low rank: first row of t
    int* lr = nullptr;         // low-rank blocks with rank > 0
    int* eptr = nullptr;       // per leaf row cluster: blocks covering it (CSR)
    int* eblk = nullptr;
    int* eroff = nullptr;      // row offset of the leaf inside the block
    double2 *D64 = nullptr, *U64 = nullptr, *V64 = nullptr, *xt64 = nullptr, *t64 = nullptr;
    float2 *D32 = nullptr, *U32 = nullptr, *V32 = nullptr, *xt32 = nullptr, *t32 = nullptr;
};

struct Ctx {
    std::string err;
    HmDev hm;
    Prof prof;
    int device = 0;
    // problem
    int nb[3] = {0, 0, 0};      // body grid
    int ne[3] = {0, 0, 0};      // extended grid
    int off[3] = {0, 0, 0};     // body offset inside ext
    double h = 0, origin[3] = {0, 0, 0};
    double freq = 0, omega = 0, k0 = 0;
    int64_t n_b = 0, n_e = 0;
    int m_f = 0, m_n = 0, s = 3;
    int64_t N = 0;
    int max_rhs = 16;
    int precisions = 3;
    vsie_options opts{};
    FFTPlan plan[3];            // radices up to 8 (FP64 kernels, spectra set-up)
    FFTPlan plan16[3];          // radices up to 16 (FP32 convolution kernels)
    FFTPlan plan3h, plan3h16;   // length L3 / 2 (twiddle steps into the L3 table), L3 even
    int L[3] = {0, 0, 0}, Lh[3] = {0, 0, 0};   // FFT lengths and octant sizes (L/2 + 1)
    // host copies (for save / get_parts / setup bookkeeping)
    std::vector<double> eps_r, sigma;
    std::vector<std::complex<double>> hW, hPreVal, hZnn, hU, hV, hZff, hTT[3][4];
    std::vector<int32_t> hBase, hPreCol;
    std::vector<int64_t> hPreRow;
    std::vector<std::complex<double>> hPreValRows, hPreValT;   // compressed-row orders
    std::vector<int64_t> sc_src;       // scatter CSR entry -> index into hW
    int aca_rank = 0;
    int tt_rank[3][3] = {{0}};
    std::vector<double> port_len;      // per port: edge length (far ports first)
    std::vector<int64_t> port_row;     // per port: unknown index
    int nloads = 0;                    // lumped loads on port edges (ports.cu)
    int64_t* load_rows = nullptr;      // device: loaded unknowns
    double2* load_d64 = nullptr;       // device: i omega eps0 Z_L l^2 per load
    float2* load_d32 = nullptr;
    // device index structures (precision independent)
    uint8_t* mask = nullptr;           // n_b material flags
    int32_t* line_ptr = nullptr;       // per ext line (i2,i3): CSR of active voxels
    int32_t* line_i1 = nullptr;        // active entries: i1 within the line
    int32_t* line_cidx = nullptr;      // active entries: compact index
    int64_t nact = 0;                  // number of active voxels
    int32_t* sc_ptr = nullptr;         // scatter CSR rows: 3 * nact + 1
    int32_t* sc_col = nullptr;         // scatter CSR columns (RWG index)
    int64_t sc_nnz = 0;
    int32_t* W_cidx = nullptr;         // m_n x s^3 compact index of each stencil voxel
    // precorrection, row-compressed CSR (only rows with entries)
    int64_t pre_nr = 0;                // non-empty body-unknown rows
    int32_t* pre_rows = nullptr;       // their indices a * n_b + v
    int64_t* pre_ptr = nullptr;        // pre_nr + 1
    int32_t* pre_col = nullptr;        // RWG index
    int64_t pre_nnz = 0;
    int64_t preT_nr = 0;               // transposed form: rows are RWG indices
    int32_t* preT_rows = nullptr;
    int64_t* preT_ptr = nullptr;
    int32_t* preT_col = nullptr;       // body unknown index (a * n_b + v)
    int32_t* body_lines = nullptr;     // flags per ext line: 1 body, 2 active, 3 both
    OpData<float> f32;
    OpData<double> f64;
    std::vector<void*> allocs;         // every device allocation (freed at destroy)
    void* conv_work = nullptr;         // FFT work buffers of the convolution (both precisions:
    size_t conv_work_bytes = 0;        // FP32 and FP64 matvecs never run at the same time)
    // solver scratch (FP64)
    double2* kr_V = nullptr;           // Krylov basis
    double2* kr_Z = nullptr;           // flexible directions (FP32 stored as float2)
    size_t kr_bytes = 0;
    bool owns_all = true;
    double2* dZff_in = nullptr;        // far-far block handed over on the device (FP64)
    bool pc_ready = false;             // block preconditioner built
    bool pc_tc = false;                // FP32 Z_ff^-1 row-major, applied on the tensor cores
    int64_t pc_ld = 0;                 // its row pitch (complex values, even)
    alignas(64) unsigned char pc_map[128] = {0};   // its TMA tensor map (CUtensorMap)
    int* tc_err = nullptr;             // device flag: a bounded wait of the tensor-core kernel ran out
    float* pc_bprep = nullptr;         // prepared B' chunks of the tensor-core product
    size_t pc_bprep_elems = 0;
    int num_sms = 152;                 // multiprocessors of the context's device
    void* net = nullptr;               // attached learned body preconditioner (not owned)
    float* net_mat = nullptr;          // 2 x n_b: (eps_r - 1) / 50, sigma
    double* net_part = nullptr;        // reduction partials of the network's input scale
    float* net_scale = nullptr;        // per RHS: RMS of the Jacobi-scaled body residual
    double* rwg_geo = nullptr;         // device, per RWG (far first, then near): per half
                                       // T+, T- the 3 vertices, the free vertex, s l / 2
                                       // (26 doubles); set by vsie_setup, else null
    vsie_parts parts_view{};           // filled by vsie_get_parts
    std::vector<std::complex<double>> hZff_copy;
    std::vector<std::complex<double>> hZnn_direct;   // set-up only: Z_nn for the preconditioner
};

// RAII scope charging kernel launches to a profiling group.
struct ProfScope {
    Ctx& c;
    int prev;
    cudaStream_t st;
    cudaEvent_t e0 = nullptr;
    ProfScope(Ctx& c_, int g, cudaStream_t s, double alg_bytes = 0.0) : c(c_), prev(c_.prof.group), st(s) {
        c.prof.group = g;
        if (c.prof.on) {
            cudaEventCreate(&e0);
            cudaEventRecord(e0, st);
            c.prof.alg_bytes[g] += alg_bytes;
        }
    }
    ~ProfScope() {
        if (c.prof.on && e0) {
            cudaEvent_t e1;
            cudaEventCreate(&e1);
            cudaEventRecord(e1, st);
            c.prof.ev[c.prof.group].push_back({e0, e1});
        }
        c.prof.group = prev;
    }
};
inline void prof_count(Ctx& c, int n) { c.prof.launches[c.prof.group] += n; }

template <typename R> OpData<R>& data(Ctx& c);
template <> inline OpData<float>& data<float>(Ctx& c) { return c.f32; }
template <> inline OpData<double>& data<double>(Ctx& c) { return c.f64; }

// ----------------------------------------------------------------- helpers
#define VSIE_CUDA(call)                                                            \
    do {                                                                           \
        cudaError_t e_ = (call);                                                   \
        if (e_ != cudaSuccess) {                                                   \
            throw ::vsie::Error(VSIE_ECUDA, std::string(#call) + ": " +            \
                                cudaGetErrorString(e_));                           \
        }                                                                          \
    } while (0)

struct Error {
    vsie_status st;
    std::string msg;
    Error(vsie_status s, std::string m) : st(s), msg(std::move(m)) {}
};

void* dalloc(Ctx& c, size_t bytes);  // cudaMalloc tracked in c.allocs, throws ENOMEM
void set_global_err(const std::string& m);  // message for vsie_last_error(NULL)
void convert_to_f32(const double2* a, float2* b, size_t n);

// launchers (defined in conv.cu / surface.cu)
template <typename R>
void conv_apply(Ctx& c, int p, const cx<R>* X, int64_t ldx, cx<R>* Y, int64_t ldy,
                cudaStream_t st);
template <typename R>
void surface_apply(Ctx& c, int p, const cx<R>* X, int64_t ldx, cx<R>* Y, int64_t ldy,
                   cudaStream_t st);
template <typename R>
void surface_pre(Ctx& c, int p, const cx<R>* X, int64_t ldx, cudaStream_t st);
template <typename R>
void conv_set_attrs();
template <typename R>
void conv_autotune(Ctx& c);
void build_block_precond(Ctx& c);
// lumped loads (ports.cu): Y += diag(loads) X on the loaded rows
template <typename R>
void apply_loads(Ctx& c, int p, const cx<R>* X, int64_t ldx, cx<R>* Y, int64_t ldy, cudaStream_t st);
// FP32 row-panel storage of the dense far blocks (gemm.cu): C = P B for
// N right-hand sides; to_panel converts a column-major M x K matrix (lda = M,
// freed) into a new panel allocation; from_panel writes it back column-major.
void gemm_panel(Ctx& c, int M, int N, int K, const float2* P, const float2* B, int64_t ldb, float2* C,
                int64_t ldc, cudaStream_t st);
float2* to_panel(Ctx& c, float2* A, int M, int K);
// Tensor-core product (tcgemm.cu): C = A B for row-major FP32 complex A (M x K,
// row pitch lda even) described by the TMA tensor map `map` (tc_make_map), N
// columns of B and C.  tc_make_map returns false if the map cannot be encoded.
bool tc_make_map(void* map, const float2* A, int M, int K, int64_t lda);
void tc_gemm(Ctx& c, const void* map, int M, int N, int K, const float2* B, int64_t ldb, float2* C, int64_t ldc,
             cudaStream_t st);
// Y = Z_ff^-1 X on the far rows with the FP32 block preconditioner (precond.cu)
void apply_far_inverse32(Ctx& c, int p, const float2* X, int64_t ldx, float2* Y, int64_t ldy, cudaStream_t st);
void from_panel(const float2* P, int M, int K, float2* A);
// learned body preconditioner (nettrain.cu): Y = M X with the surface blocks of
// the block preconditioner and the attached network on the body
void apply_learned_precond(Ctx& c, int p, const float2* X, int64_t ldx, float2* Y, int64_t ldy,
                           cudaStream_t st);
template <typename R>
void apply_block_precond(Ctx& c, int p, const cx<R>* X, int64_t ldx, cx<R>* Y, int64_t ldy,
                         cudaStream_t st);
template <typename R>
void upload_twiddles(Ctx& c);

enum GemmOp { OP_N = 0, OP_T = 1, OP_H = 2, OP_R = 3 };  // R = conj, no transpose

// C_b = alpha * op(A_b) * B_b + beta * C_b, b in [0, batch); optional masks:
// maskB[k + K * n] gates B elements (zero when 0), maskC[m + M * n] gates the
// update of C elements.  Column-major, complex.
template <typename R>
void cgemm(Ctx& c, GemmOp opA, int M, int Nn, int K, cx<R> alpha, const cx<R>* A, int64_t lda,
           int64_t sA, const cx<R>* B, int64_t ldb, int64_t sB, cx<R> beta, cx<R>* C,
           int64_t ldc, int64_t sC, int batch, const uint8_t* maskB, const uint8_t* maskC,
           cudaStream_t st);

template <typename R>
void cgemm2(Ctx& c, GemmOp opA, GemmOp opB, int M, int Nn, int K, cx<R> alpha, const cx<R>* A,
            int64_t lda, int64_t sA, const cx<R>* B, int64_t ldb, int64_t sB, cx<R> beta,
            cx<R>* C, int64_t ldc, int64_t sC, int batch, const uint8_t* maskB,
            const uint8_t* maskC, cudaStream_t st);

// volume spectra set-up (green.cu)
template <typename R>
void build_spectra(Ctx& c);

}  // namespace vsie
