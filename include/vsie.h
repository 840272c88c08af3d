/*
 * vsie.h - C ABI of libvsie, a GB300 (sm_103a) implementation of the hybrid
 * volume-surface integral equation (hybrid-VSIE) matrix-vector product and the
 * GMRES that applies it (Giannakopoulos et al., "A hybrid volume-surface
 * integral equation method for rapid electromagnetic simulations in MRI").
 *
 * The system solved is Eq. (hvsie) of the paper,
 *
 *     [ Z_ff    Z_fn^T  Z_fb^T ] [ j_f ]   [ v_f ]
 *     [ Z_fn    Z_nn    Z_nb^T ] [ j_n ] = [ v_n ]
 *     [ Z_fb    Z_nb    Z_bb   ] [ j_b ]   [  0  ]
 *
 * in its compressed form Eq. (hvsie_disc): far conductors (shield, bore) j_f,
 * near conductors (coils) j_n, body polarisation currents j_b.  Z_bb and the
 * near block are applied by the precorrected FFT on an extended voxel grid
 * (Sec. II.C, III), Z_fn by its ACA factors U V^H (Sec. III), the far coupling
 * Z_fb by its tensor trains with Eq. (mvp) and Eq. (tmvp), and Z_ff densely or
 * as a hierarchical matrix whose admissible blocks are ACA factors (Sec. II.B).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Unknown vector of length N = m_f + m_n + 3 * n_b, ordered [j_f; j_n; j_b].
 *    j_b is component-major: j_b[a * n_b + v], a in {x, y, z}, body voxel
 *    v = i1 + n1 * (i2 + n2 * i3) (i1 fastest, the column-major order of
 *    Eq. (mvp)).
 *  - Complex numbers are interleaved (re, im): double2 for VSIE_C128, float2
 *    for VSIE_C64.  Blocks of p right-hand sides are column-major with a
 *    leading dimension (in complex elements) >= N.
 *  - Voxels whose material has chi = eps_r - 1 - i sigma / (omega eps0) = 0
 *    (vacuum) carry identity rows and columns: their output equals their input.
 *  - Device pointers are owned by the caller (for example torch tensors); the
 *    library never frees caller memory.  A context owns all its own device
 *    allocations and frees them in vsie_destroy.
 *  - Work is enqueued on the caller's stream and is asynchronous unless stated.
 *  - A context is not thread-safe: use one per host thread and stream.
 *  - No exceptions or aborts cross the ABI.  Every call returns a status; the
 *    message of the last failure is returned by vsie_last_error.
 */
#ifndef VSIE_H
#define VSIE_H

#include <stdint.h>

#if defined(__GNUC__)
#define VSIE_API __attribute__((visibility("default")))
#else
#define VSIE_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct vsie_ctx vsie_ctx;
typedef struct CUstream_st* vsie_stream; /* a cudaStream_t; NULL = legacy default stream */

typedef enum {
    VSIE_OK = 0,
    VSIE_EINVAL = 1,       /* invalid argument (null pointer, size, mesh, grid) */
    VSIE_ENOMEM = 2,       /* device or host allocation failed */
    VSIE_ECUDA = 3,        /* a CUDA runtime call failed */
    VSIE_ENOCONV = 4,      /* iterative solver hit maxit; X holds the last iterate */
    VSIE_EBREAKDOWN = 5,   /* non-finite values met (NaN/Inf in data or iterate) */
    VSIE_ETIMEOUT = 6,     /* a bounded device wait ran out */
    VSIE_EUNSUPPORTED = 7  /* valid but unsupported request (e.g. FFT length) */
} vsie_status;

enum { VSIE_C128 = 0, VSIE_C64 = 1 };

/* Uniform voxel grid: n[0] x n[1] x n[2] voxels of edge h (metres); voxel
 * (0,0,0) is centred at origin. */
typedef struct {
    int32_t n[3];
    double h;
    double origin[3];
} vsie_grid;

/* Triangle mesh (metres): xyz[3*nverts], tri[3*ntris] (vertex ids),
 * ports[2*nports] (vertex pairs naming interior port edges). */
typedef struct {
    int32_t nverts;
    const double* xyz;
    int32_t ntris;
    const int32_t* tri;
    int32_t nports;
    const int32_t* ports;
} vsie_mesh;

/* Set-up options.  Zero-initialise and override; zeros select the defaults. */
typedef struct {
    int32_t ext_n[3];      /* extended pFFT grid (0 = the body grid)                    */
    int32_t ext_offset[3]; /* body grid offset inside the extended grid                 */
    int32_t stencil;       /* pFFT expansion stencil s (odd; default 3)                 */
    int32_t near_radius;   /* precorrection radius in voxels (default s + 1)            */
    double colloc_rfac;    /* collocation sphere radius = rfac * s * h / 2 (default 2)  */
    double tt_tol;         /* TT tolerance of the far coupling (default 1e-6)           */
    double aca_tol;        /* ACA tolerance of the near-far block (default 1e-6)        */
    int32_t max_rhs;       /* largest p passed to vsie_matvec / vsie_solve (default 16) */
    int32_t precisions;    /* bit mask (1 << VSIE_C128) | (1 << VSIE_C64); default both */
    int32_t far_hmatrix;   /* far-far block Z_ff (vsie_setup only): 0 = hierarchical when
                              m_f >= 8192, else dense; 1 = hierarchical; -1 = dense     */
    int32_t hm_leaf;       /* H-matrix leaf cluster size, <= 256 (default 128)          */
    double hm_eta;         /* H-matrix admissibility min(diam) <= eta dist (default 1)  */
    int32_t dense_gemm;    /* FP32 product with the preconditioner's dense far-block
                              inverse: 0 = tensor cores (tcgen05, split TF32), 1 = SIMT  */
    int32_t reserved;      /* zero                                                      */
} vsie_options;

/* Compressed operator parts, for vsie_create.  All arrays are host memory,
 * complex interleaved (double2), column-major unless stated.  Sizes:
 *   W          [m_n][3 s^3]  projection weights of each near RWG, index
 *                            b * s^3 + qx + s*(qy + s*qz) (row per RWG)
 *   base       [m_n][3]      lowest-corner voxel (ext grid) of each stencil
 *   pre_*      CSR of the precorrection (Z form) with 3 n_b rows (body unknowns)
 *              and m_n columns: rowptr[3 n_b + 1], col[nnz], val[nnz]
 *   Znn        m_n x m_n     near block with the grid part folded out
 *   U, V       m_n x k, m_f x k   U V^H ~= Z_fn  (k = aca_rank, may be 0)
 *   Zff        m_f x m_f
 *   tt_rank    [3][3]        (r1, r2, r3) per component
 *   tt_core    [3][4]        G1 (n1 x r1), G2 (r1 x n2 x r2), G3 (r2 x n3 x r3),
 *                            G4 (r3 x m_f), column-major (first index fastest)
 * m_n = 0 or m_f = 0 drop the corresponding blocks. */
typedef struct {
    int32_t m_f, m_n, stencil;
    const double* W;
    const int32_t* base;
    int64_t pre_nnz;
    const int64_t* pre_rowptr;
    const int32_t* pre_col;
    const double* pre_val;
    const double* Znn;
    int32_t aca_rank;
    const double* U;
    const double* V;
    const double* Zff;
    int32_t tt_rank[3][3];
    const double* tt_core[3][4];
} vsie_parts;

/* Solver options for vsie_solve (zero-initialise; zeros select defaults). */
typedef struct {
    int32_t mode;       /* 0 = plain FP64 GMRES; 1 = FP32 inner GMRES with FP64 refinement  */
    int32_t restart;    /* GMRES restart length m (default 50)                            */
    int32_t maxit;      /* total inner iteration cap per RHS (default 2000)               */
    double inner_tol;   /* mode 1: relative tolerance of each inner solve (default 1e-4)  */
    int32_t max_outer;  /* mode 1: refinement steps cap (default 20)                      */
    int32_t precond;    /* right preconditioner: 0 = block (inverses of the two surface
                           blocks, inverse body diagonal; default), 1 = none, 2 = block
                           with the attached network on the body (vsie_net_attach),
                           which makes the inner solve flexible GMRES (FGMRES)         */
} vsie_solve_opts;

typedef struct {
    int32_t iters[64];      /* inner iterations per RHS (first 64 RHS)                   */
    double relres[64];      /* final true relative residual ||b - Z x|| / ||b|| (FP64)   */
    int32_t outer;          /* refinement steps taken (mode 1)                           */
    int32_t matvecs64;      /* FP64 block operator applications (each over the p columns) */
    int32_t matvecs32;      /* FP32 block operator applications (each over the p columns) */
    double seconds;         /* wall time of the solve                                     */
} vsie_solve_info;

/* Message of the last failure on ctx (or of the last failed context-less call
 * when ctx is NULL).  The pointer stays valid until the next call. */
VSIE_API const char* vsie_last_error(const vsie_ctx* ctx);

/* Library version string. */
VSIE_API const char* vsie_version(void);

/* Full set-up from geometry (Sec. III): body grid and material maps
 * (eps_r, sigma: n_b host doubles each, S/m), near conductors `coil` and far
 * conductors `shield` (either may be NULL), frequency in Hz.  Builds RWG
 * functions, the Green spectra of the extended grid, the pFFT projection and
 * precorrection, the dense near block, the ACA factors of Z_fn, Z_ff (dense, or
 * hierarchical with ACA blocks at aca_tol: see far_hmatrix) and the TT of Z_fb
 * (ACA matrix cross over the (voxel | far RWG) unfolding, then TT-SVD of the
 * voxel factor).  With a hierarchical Z_ff the dense block is kept only while
 * the preconditioner is built: vsie_get_parts and vsie_save then return
 * EUNSUPPORTED, and plain FP64 solves (mode 0, which need the FP64 inverse of
 * the dense block) return EUNSUPPORTED.  Synchronous; uses the current device.
 * Returns EINVAL for malformed meshes/grids or stencils leaving the extended
 * grid, ENOMEM/ECUDA on device failures.  *out is set only on success. */
VSIE_API vsie_status vsie_setup(const vsie_grid* body, const double* eps_r, const double* sigma,
                       const vsie_mesh* coil, const vsie_mesh* shield, double freq_hz,
                       const vsie_options* opts, vsie_ctx** out);

/* Create a context from precomputed compressed parts (for example loaded from
 * disk, or produced by another implementation).  Same body/material/frequency
 * meaning as vsie_setup; parts may be NULL (volume operator only).  The Green
 * spectra are computed here.  Synchronous. */
VSIE_API vsie_status vsie_create(const vsie_grid* body, const double* eps_r, const double* sigma,
                        double freq_hz, const vsie_options* opts, const vsie_parts* parts,
                        vsie_ctx** out);

/* Sizes of the unknown vector. Any output pointer may be NULL. */
VSIE_API vsie_status vsie_sizes(const vsie_ctx* ctx, int64_t* N, int64_t* m_f, int64_t* m_n,
                       int64_t* n_b);

/* Y = Z X for p right-hand sides (Eq. hvsie_disc).  X, Y: device pointers,
 * column-major N x p with leading dimensions ldx, ldy (complex elements);
 * precision VSIE_C128 (double2) or VSIE_C64 (float2).  X and Y must not
 * overlap.  1 <= p <= opts.max_rhs.  Asynchronous on `stream`. */
VSIE_API vsie_status vsie_matvec(vsie_ctx* ctx, int32_t p, const void* X, int64_t ldx, void* Y,
                        int64_t ldy, int32_t precision, vsie_stream stream);

/* Delta-gap right-hand sides i omega eps0 V l_m of the listed ports (indices
 * into the concatenation [shield ports; coil ports]) into B (device, double2,
 * column-major N x nports, leading dimension ldb), one column per port. */
VSIE_API vsie_status vsie_rhs_ports(vsie_ctx* ctx, int32_t nports, const int32_t* ports, double V,
                           void* B, int64_t ldb, vsie_stream stream);

/* Right-hand side of Eq. (hvsie) for an incident plane wave
 * E_inc(r) = e0 exp(-i k0 khat . r) (Sec. II.A: the equivalent currents are
 * driven by the incident field; time convention exp(+i omega t)), written to one
 * column B (device, double2, N values):
 *   conductor rows  i omega eps0 \int f_m . E_inc dS  (6-point Dunavant rule per
 *                   triangle; the delta-gap port is the impressed-field case of
 *                   the same row),
 *   body rows       i omega eps0 h^3 E_inc(r_p), component-major, on material
 *                   voxels; 0 on vacuum voxels.
 * k_hat (host, 3 doubles) is normalised here; e0 (host, 3 doubles, V/m, real
 * linear polarisation) must be orthogonal to k_hat (EINVAL otherwise).  The
 * conductor rows need the meshes given to vsie_setup: a context created from
 * parts or loaded from a file that has conductors returns EUNSUPPORTED.
 * Asynchronous on `stream`. */
VSIE_API vsie_status vsie_rhs_planewave(vsie_ctx* ctx, const double k_hat[3], const double e0[3], void* B,
                                        vsie_stream stream);

/* One right-hand side with several ports driven at once (Sec. V: a coil array
 * driven in a chosen mode, e.g. the circularly polarised mode of an n-loop array,
 * v_k = exp(-i 2 pi k / n) for loop k): port ports[i] (index into [shield ports;
 * coil ports]) carries the delta-gap voltage v[2 i] + i v[2 i + 1] volts, so its
 * row is i omega eps0 v_i l; every other entry of B (device, double2, N values) is
 * zero.  EINVAL for bad indices, a port listed twice or non-finite voltages.
 * Asynchronous on `stream` after a synchronous upload of the nports values; it
 * returns once the entries are written. */
VSIE_API vsie_status vsie_rhs_drive(vsie_ctx* ctx, int32_t nports, const int32_t* ports, const double* v, void* B,
                                    vsie_stream stream);

/* Lumped loads (Sec. IV.B, V: tuning and matching elements of the coil ports):
 * impedance z_load[2 i] + i z_load[2 i + 1] ohms in series with the edge of port
 * ports[i] (index into [shield ports; coil ports]).  Its voltage drop enters the
 * port row, so the operator's diagonal entry of that edge gains
 * i omega eps0 Z_L l^2 (l the edge length); vsie_matvec and vsie_solve apply it
 * in both precisions.  The block preconditioner is not rebuilt.  Replaces the
 * previous loads; nloads = 0 removes them; vsie_save does not store them.  EINVAL for bad indices, a port
 * listed twice or non-finite values.  Synchronous. */
VSIE_API vsie_status vsie_set_loads(vsie_ctx* ctx, int32_t nloads, const int32_t* ports, const double* z_load);

/* Network parameters of the listed ports (Sec. V): X (device, double2, N x nports,
 * leading dimension ldx) holds the solutions with port j driven by 1 V
 * (vsie_rhs_ports with V = 1) and the others shorted.  The current through port
 * edge i is I_ij = x_i l_i, so the admittance matrix is Y = I (siemens); the
 * impedance matrix Z = Y^-1 (ohms) and the scattering matrix
 * S = (Z - z0)(Z + z0)^-1 for the reference impedance z0 (ohms).  Y, Z, S (host,
 * any may be NULL): nports x nports complex, column-major, interleaved (re, im).
 * EBREAKDOWN when Y or Z + z0 is singular.  Synchronous. */
VSIE_API vsie_status vsie_port_network(vsie_ctx* ctx, int32_t nports, const int32_t* ports, const void* X,
                                       int64_t ldx, double z0, double* Y, double* Z, double* S);

/* Solve Z X = B for p right-hand sides to relative FP64 residual tol (Sec. III.A:
 * GMRES with restart; x0 = 0).  B, X: device double2 (C128), column-major N x p.
 * mode 0: every matvec, orthogonalisation and Givens update in FP64.
 * mode 1: iterative refinement: FP64 outer residual r = B - Z X, inner GMRES on
 * the FP32 operator with an FP32 basis and FP32 Gram-Schmidt (FP64 across thread
 * blocks), FP64 Givens on the host.  precond = 2 makes the solve flexible GMRES
 * (the network's output depends on its input).  Synchronous with respect to
 * `stream`.  info (host) may be NULL.  Returns ENOCONV when any RHS misses tol
 * (X then holds the last iterate and info its residual). */
VSIE_API vsie_status vsie_solve(vsie_ctx* ctx, int32_t p, const void* B, int64_t ldb, void* X,
                       int64_t ldx, double tol, const vsie_solve_opts* opts,
                       vsie_solve_info* info, vsie_stream stream);

/* Uneven batch (many independent problems of different sizes): solve
 * ctxs[i] Z_i X_i = B_i (p[i] columns, leading dimensions ldb[i], ldx[i], device
 * double2) for i < nctx with the options and tolerance of vsie_solve.  Up to
 * nthreads host threads (0: 8) each take the next context and solve it on a
 * stream of their own, so the kernels of small problems overlap on the GPU.
 * Every context may appear once, and with precond = 2 no two contexts may share
 * a network (EINVAL).  info and status (nctx entries each, host)
 * may be NULL; returns VSIE_OK when every solve did, else the first failing
 * status.  Synchronous. */
VSIE_API vsie_status vsie_solve_batch(int32_t nctx, vsie_ctx* const* ctxs, const int32_t* p,
                                      const void* const* B, const int64_t* ldb, void* const* X,
                                      const int64_t* ldx, double tol, const vsie_solve_opts* opts,
                                      vsie_solve_info* info, vsie_status* status, int32_t nthreads);

/* Profiling.  vsie_profile(ctx, 1) clears the counters and starts recording a
 * CUDA event pair around every kernel group launched by calls on the context
 * (0 stops recording; launch counts are always kept).  vsie_profile_query
 * synchronises the device and returns, for a group, the summed event time in
 * ms, the number of kernel launches and the algorithmic bytes moved (defined
 * for groups 0 and 7 only: 54 complex values per extended-grid voxel and RHS
 * plus the spectrum octants).  Groups: 0 FFT convolution (K1) in FP32 (C64),
 * 1 pFFT projection and interpolation, 2 precorrection, 3 dense and low-rank
 * surface blocks, 4 TT chain, 5 Krylov vector kernels, 6 preconditioner, 7 FFT
 * convolution in FP64 (C128); group -1 returns the launches of all groups. */
VSIE_API vsie_status vsie_profile(vsie_ctx* ctx, int32_t enable);
VSIE_API vsie_status vsie_profile_query(vsie_ctx* ctx, int32_t group, double* ms, int64_t* launches,
                                        double* alg_bytes);

/* Body block only, y_b = Z_bb x_b, without allocating anything (this library
 * has no counterpart of it in the paper).  For callers that cannot allocate
 * device memory while the operator runs (a fixed memory pool that must not
 * grow, a real-time loop that may not wait on the allocator, a host runtime
 * that owns all device memory itself).  X and Y hold
 * p body vectors of 3 n_b complex values each (component-major, device,
 * leading dimensions >= 3 n_b).  Vacuum voxels return their input.
 * The FFT work space comes from one file-scope device array of 32 MiB that
 * every GPU loading the library keeps until exit; requests needing more
 * (p * 3 * n3 * (n2 + L2) * L1 complex values, L = FFT lengths of the context)
 * return VSIE_EINVAL.  The first call on a device looks up that array's device
 * address with the device current; make that first call before any stream
 * capture.  The address is kept for the life of the process, so resetting a
 * device (cudaDeviceReset) after its first call is not supported.  All calls on
 * a device share its copy of the array, which keeps the last call's contents;
 * nothing in it needs to start at zero.  Calls that overlap on the same GPU
 * (for example on two streams, or solves of vsie_solve_batch running on their
 * worker threads) race on it.  Asynchronous on `stream`. */
VSIE_API vsie_status vsie_volume_matvec_static(vsie_ctx* ctx, int32_t p, const void* X, int64_t ldx,
                                               void* Y, int64_t ldy, int32_t precision,
                                               vsie_stream stream);

/* Persistence of a context's operator (Sec. VI: compressed coupling matrices
 * stored and reused).  vsie_save writes the body grid, materials, frequency,
 * options, every part of vsie_parts (the far block copied from the device) and
 * the port table to a versioned binary file at `path`; vsie_load reads it back,
 * checks every array size against the header, and recreates the context with
 * vsie_create (set-up integrals are not recomputed).  EINVAL for unreadable,
 * foreign or truncated files; the caller owns the new context. */
VSIE_API vsie_status vsie_save(const vsie_ctx* ctx, const char* path);
VSIE_API vsie_status vsie_load(const char* path, vsie_ctx** out);

/* Copy the context's parts to host arrays owned by the context (valid until
 * vsie_destroy); pointers in *parts refer to that storage. */
VSIE_API vsie_status vsie_get_parts(vsie_ctx* ctx, vsie_parts* parts);

/* ---------------------------------------------------------------------------
 * Learned body preconditioner (not in the paper; cf. the preconditioning of the
 * coupled system suggested in Sec. VI).  A 3D U-Net: 4 levels with 16/32/64/64
 * channels, 3x3x3 convolutions (zero padding), ReLU, 2x2x2 average pooling,
 * nearest x2 upsampling, skips concatenated after the upsampled tensor, and a
 * linear 1x1x1 head; 15 layers e1a 8->16, e1b 16->16, e2a 16->32, e2b 32->32,
 * e3a 32->64, e3b 64->64, ba 64->64, bb 64->64, d3a 128->64, d3b 64->64,
 * d2a 96->32, d2b 32->32, d1a 48->16, d1b 16->16, head 16->6 (1x1x1).
 * Tensors: FP32, channel-major (C, D, H, W), W fastest, D, H, W multiples of 8.
 * Parameters: FP32 master values, packed layer by layer as the weights
 * (Cout, Cin, k, k, k) followed by the biases (Cout); the kernels use BF16
 * copies of the weights and accumulate in FP32.  Input channels: re/im of the
 * three components of the Jacobi-scaled body residual divided by its RMS, then
 * (eps_r - 1) / 50 and sigma (S/m); output: the 6-channel correction.
 * All device pointers belong to the caller.  Errors: vsie_net_last_error. */
typedef struct vsie_net vsie_net;

/* He-normal weights from `seed`, zero biases, Adam state zero. */
VSIE_API vsie_status vsie_net_create(uint64_t seed, vsie_net** out);
VSIE_API vsie_status vsie_net_num_params(const vsie_net* net, int64_t* n);
/* Host copies of the n packed parameters (n must equal vsie_net_num_params). */
VSIE_API vsie_status vsie_net_set_params(vsie_net* net, const float* host, int64_t n);
VSIE_API vsie_status vsie_net_get_params(vsie_net* net, float* host, int64_t n);
/* y (6 x D x H x W, device) = net(x) (x: 8 x D x H x W, device).  Async on stream. */
VSIE_API vsie_status vsie_net_forward(vsie_net* net, int32_t D, int32_t H, int32_t W, const float* x,
                                      float* y, vsie_stream stream);
/* Gradients of sum(dy * net(x)): parameters to grad_host (packed like the
 * parameters; may be NULL) and the input gradient to dx (device, 8 x D x H x W;
 * may be NULL).  Synchronous. */
VSIE_API vsie_status vsie_net_backward(vsie_net* net, int32_t D, int32_t H, int32_t W, const float* x,
                                       const float* dy, float* grad_host, float* dx,
                                       vsie_stream stream);
/* One training step: loss = mean((net(x) - target)^2) over all 6 D H W
 * entries, its gradient, one Adam update (lr; beta 0.9, 0.999; eps 1e-8).
 * Returns the loss before the update in *loss (may be NULL).  Synchronous. */
VSIE_API vsie_status vsie_net_step(vsie_net* net, int32_t D, int32_t H, int32_t W, const float* x,
                                   const float* target, double lr, double* loss, vsie_stream stream);
/* Train on pairs the context's own operator generates: per step a seeded
 * smooth random body current e (material voxels), r = Z_bb e by the FP32
 * operator, input from the Jacobi-scaled r, target (e - D^-1 r) / s; Adam with
 * the learning rate decaying linearly from lr to lr / 10 over the steps.  Writes
 * `steps` losses to losses_host (may be NULL).  Synchronous. */
VSIE_API vsie_status vsie_net_train(vsie_ctx* ctx, vsie_net* net, int32_t steps, double lr,
                                    uint64_t seed, float* losses_host, vsie_stream stream);
/* Use `net` (not owned; NULL detaches) on the body block when a solve asks for
 * precond = 2. */
/* Y = M X for p columns with the FP32 (C64) right preconditioner of a solve:
 * kind 0 the block preconditioner, kind 2 the block preconditioner with the
 * attached network on the body.  X, Y: device float2, N x p, must not overlap.
 * Asynchronous on `stream`. */
VSIE_API vsie_status vsie_precond_apply(vsie_ctx* ctx, int32_t p, const void* X, int64_t ldx, void* Y,
                                        int64_t ldy, int32_t kind, vsie_stream stream);
VSIE_API vsie_status vsie_net_attach(vsie_ctx* ctx, vsie_net* net);
VSIE_API const char* vsie_net_last_error(const vsie_net* net);
VSIE_API void vsie_net_destroy(vsie_net* net);

VSIE_API void vsie_destroy(vsie_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* VSIE_H */
