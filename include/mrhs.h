/*
 * mrhs.h - C ABI of the GB300 (sm_103a) multiple-right-hand-side setup of
 * two-level DD-alpha-AMG for the Wilson-clover Dirac operator
 * (Richtmann, Heybrock, Wettig, arXiv:1601.03184).
 *
 * Every step of the setup runs in the library's own CUDA kernels. The calls
 * below are the boundary: plain pointers and sizes, no C++ or torch types.
 *
 * General rules for every call
 *  - Return value: MRHS_OK (0) or a negative mrhs_status. No exception and no
 *    abort crosses this boundary; mrhs_last_error(ctx) holds the message of
 *    the last failure on that context (mrhs_last_error(NULL): failures of
 *    mrhs_create).
 *  - Host pointers are owned by the caller and read or written only during
 *    the call. Device pointers are owned by the caller, must be 16-byte
 *    aligned, and are read/written in stream order on the context's stream
 *    (the call may return before the GPU has finished; mrhs_sync waits).
 *    Every call checks the memory type of the caller's pointers before any
 *    launch or copy (cudaPointerGetAttributes): host memory or another GPU's
 *    memory where a device field of the context's GPU is expected, or device
 *    memory where a host array is expected, returns MRHS_ERR_ARG. Managed
 *    memory is accepted for both.
 *    Everything the library allocates is freed by mrhs_destroy.
 *  - Sites: canonical index s = x + Lx*(y + Ly*(z + Lz*t)); spinor component
 *    c = 3*spin + colour; chirality h = 0 for spins 0,1 (gamma_5 = +1), h = 1
 *    for spins 2,3, in the chiral gamma basis gamma_k = [[0,-i sigma_k],
 *    [i sigma_k,0]] (mu = k-1 = 0,1,2), gamma_4 = [[0,1],[1,0]] (mu = 3).
 *    Fermion fields are antiperiodic in t, periodic otherwise.
 *  - Host ("canonical") field layout: [nrhs][V][12] complex, complex128 for
 *    MRHS_F64 or complex64 for MRHS_F32 host dtypes.
 *  - Device ("interleaved") field layout: the right-hand sides are the
 *    innermost index, real parts of all nrhs then imaginary parts (the
 *    array-of-structs-of-short-vectors layout of Sec. 5 of the paper, with
 *    the vector length equal to nrhs): element (site, c, re/im, rhs) at
 *    ((site*12 + c)*2 + re/im)*nrhs + rhs, sites in the library's
 *    aggregate-major order (aggregate, then site inside it). Only the
 *    library's own pack/unpack calls write or read this order; use
 *    mrhs_field_bytes for sizes.
 *  - Coarse fields: per aggregate 2*ntv complex values (index h*ntv + j,
 *    2 N_tv coarse degrees of freedom per aggregate, Sec. 4 with Eq. 1, and
 *    Alg. 3).
 *    Host layout [nrhs][nagg][2ntv]
 *    complex; device layout ((A*2ntv + i)*2 + re/im)*nrhs + rhs.
 *  - Aggregates are lattice blocks of agg[0]x..xagg[3] sites in
 *    lexicographic block order. They are also the Schwarz domains of the SAP
 *    smoother (Sec. 2, domain size 4^4 in Sec. 7).
 */
#ifndef MRHS_H
#define MRHS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mrhs_ctx_s* mrhs_ctx;

typedef enum {
  MRHS_OK = 0,
  MRHS_ERR_ARG = -1,       /* bad pointer, enum value or parameter */
  MRHS_ERR_SHAPE = -2,     /* lattice/aggregate/ntv combination not allowed */
  MRHS_ERR_OOM = -3,       /* device or host allocation failed */
  MRHS_ERR_CUDA = -4,      /* a CUDA runtime call failed */
  MRHS_ERR_NOCONV = -5,    /* an iterative solve hit maxit before its tolerance */
  MRHS_ERR_NONFINITE = -6, /* NaN/Inf or a linearly dependent test vector */
  MRHS_ERR_STATE = -7,     /* call made before the state it needs exists */
  MRHS_ERR_TIMEOUT = -8    /* a bounded device wait (tensor-core pipeline) ran out */
} mrhs_status;

/* storage type of a field (device) or of a host array */
typedef enum { MRHS_F64 = 0, MRHS_F32 = 1, MRHS_BF16 = 2, MRHS_F16 = 3 } mrhs_dtype;

/* precision of a context: what the setup stores its test vectors, P, work
 * vectors and D_c in. FP64: all double. FP32: all float (reductions in
 * double). MIX_BF16 / MIX_FP16: test vectors and P in bf16 / fp16, smoother
 * and coarse work in float, Gram-Schmidt inner products in double. */
typedef enum { MRHS_PREC_FP64 = 0, MRHS_PREC_FP32 = 1, MRHS_PREC_MIX_BF16 = 2, MRHS_PREC_MIX_FP16 = 3 } mrhs_prec;

/* ---------------------------------------------------------------- context */

/* Create a lattice context on the current CUDA device.
 * dims: lattice extents (Lx,Ly,Lz,Lt); agg: aggregate (= Schwarz domain)
 * extents; ntv: number of test vectors N_tv (Sec. 2); prec: mrhs_prec;
 * stream: a cudaStream_t (NULL = the legacy default stream) used for every
 * later launch and copy of this context.
 * MRHS_ERR_SHAPE unless: every dims[mu] % agg[mu] == 0, every
 * dims[mu]/agg[mu] is even (red-black colouring of the domains), V < 2^30,
 * 1 <= ntv <= 6*|aggregate| and ntv <= 64. Builds the index tables. */
int mrhs_create(const int dims[4], const int agg[4], int ntv, int prec, void* stream, mrhs_ctx* out);
void mrhs_destroy(mrhs_ctx ctx);
const char* mrhs_last_error(mrhs_ctx ctx);
/* wait for all work of the context's stream; MRHS_ERR_TIMEOUT if a bounded
 * wait of a tensor-core coarse-stencil launch ran out since the last check */
int mrhs_sync(mrhs_ctx ctx);
/* out[0..7] = V, nagg, sites per aggregate, ntv, prec, device bytes held by
 * the library, number of SMs, the CUDA device the context lives on */
int mrhs_info(mrhs_ctx ctx, long long out[8]);

/* release the context's scratch buffers (work fields, Krylov bases, staging);
 * they are allocated again when a later call needs them. The setup state
 * (test vectors, P, D_c, gauge field, clover) is kept. */
int mrhs_trim(mrhs_ctx ctx);

/* bytes of a device field of nrhs right-hand sides (coarse != 0: coarse
 * field) in storage type dtype */
size_t mrhs_field_bytes(mrhs_ctx ctx, int nrhs, int dtype, int coarse);

/* Neighbour and aggregate tables, canonical order, as built on the GPU.
 * nbr [V][8]: k = 0..3 the site s + mu_hat, k = 4..7 the site s - mu_hat;
 * bit 30 set when the hop crosses the t boundary (fermion sign -1).
 * aggof [V][2]: (aggregate index, offset of s inside its aggregate, both
 * lexicographic). aggnbr [nagg][8]: aggregate +mu (k<4) and -mu (k>=4).
 * Any pointer may be NULL. */
int mrhs_get_tables(mrhs_ctx ctx, int* nbr, int* aggof, int* aggnbr);

/* ------------------------------------------------------ gauge and clover */

/* Copy the gauge field in: host U[V][4][3][3] complex128, canonical order
 * (the links U_mu(x) of the Wilson-clover operator named in Sec. 2). */
int mrhs_set_gauge(mrhs_ctx ctx, const double* U);

/* Build the clover term on the GPU (in FP64) from the gauge field:
 * A(x) = (4+m0) + (csw/2) sum_{mu<nu} i sigma_{mu nu} Fhat_{mu nu}(x),
 * sigma_{mu nu} = (i/2)[gamma_mu, gamma_nu], Fhat = (Q - Q^dag)/8 with Q the
 * four-leaf clover sum; stored as two Hermitian 6x6 blocks per site
 * (chiralities h = 0, 1). MRHS_ERR_STATE before mrhs_set_gauge. */
int mrhs_build_clover(mrhs_ctx ctx, double m0, double csw);

/* Copy the clover blocks out: host [V][2][6][6] complex128, canonical. */
int mrhs_get_clover(mrhs_ctx ctx, double* host_out);

/* ------------------------------------------------------- field transfer */

/* host canonical [nrhs][V][12] (host_dtype MRHS_F64: complex128, MRHS_F32:
 * complex64) -> device interleaved field of storage type dev_dtype. */
int mrhs_pack(mrhs_ctx ctx, const void* host, int host_dtype, void* dev, int dev_dtype, int nrhs);
/* device interleaved -> host canonical */
int mrhs_unpack(mrhs_ctx ctx, const void* dev, int dev_dtype, void* host, int host_dtype, int nrhs);
/* the same for coarse fields: host [nrhs][nagg][2ntv] */
int mrhs_pack_coarse(mrhs_ctx ctx, const void* host, int host_dtype, void* dev, int dev_dtype, int nrhs);
int mrhs_unpack_coarse(mrhs_ctx ctx, const void* dev, int dev_dtype, void* host, int host_dtype, int nrhs);

/* ------------------------------------------------------------ operators */

/* y = D x for nrhs right-hand sides at once (multi-RHS Wilson-clover
 * stencil; the operator whose linear system the solver of Sec. 1-2 targets):
 * y(x) = A(x) x(x) - 1/2 sum_mu [(1-gamma_mu) U_mu(x) x(x+mu)
 *                              + (1+gamma_mu) U_mu(x-mu)^dag x(x-mu)].
 * x, y: device interleaved fields of storage dtype (F64 computes in double,
 * the others in float). x and y must not overlap.
 * MRHS_ERR_STATE before mrhs_build_clover. */
int mrhs_apply_D(mrhs_ctx ctx, const void* x, void* y, int nrhs, int dtype);

/* y = D_B x: D with every coupling between different aggregates removed
 * (the block operator of the Schwarz smoother, Sec. 2). */
int mrhs_apply_D_block(mrhs_ctx ctx, const void* x, void* y, int nrhs, int dtype);

/* x <- SAP^n_sweeps(b, x): the Schwarz alternating procedure smoother of
 * Sec. 2 on all nrhs right-hand sides at once. One sweep = colour 0 then
 * colour 1 of the red-black domain colouring (colour = parity of the sum of
 * the aggregate coordinates); per colour r = b - D x, then on every domain
 * B of that colour n_mr minimal-residual steps on D_B e = r_B from e = 0
 * (alpha = <q,rho>/<q,q>, q = D_B rho), and x_B += e. b, x: device fields
 * of storage dtype F64 or F32. */
int mrhs_sap(mrhs_ctx ctx, const void* b, void* x, int nrhs, int dtype, int n_sweeps, int n_mr);

/* Domain solves of the SAP smoother (every use: mrhs_sap, the setup phases,
 * the V-cycle of mrhs_solve_fgmres). even_odd = 0 (default): n_mr MR steps on
 * D_B e = r_B. even_odd = 1: even-odd preconditioning (the Schur complement
 * used for the coarse grid in Sec. 4 and Eq. 1, here applied to the domain
 * solves): with E, O the sites of even and odd parity (x+y+z+t) of the domain
 * and H its hopping terms, n_mr MR steps on
 *   S e_E = r_E - H_EO A_OO^-1 r_O,   S = A_EE - H_EO A_OO^-1 H_OE,
 * from e_E = 0 (inner products over the even sites), then
 * e_O = A_OO^-1 (r_O - H_OE e_E) and x_B += e. The inverse clover term is
 * built on the first use after each mrhs_build_clover (MRHS_ERR_NONFINITE if
 * a block is singular). The even-odd form runs in the generic domain kernel
 * (one CTA per domain); the on-chip kernels serve only the plain form. It
 * needs three more FP32 work fields of the smoothed vectors and the inverse
 * clover term (about 110 GB more at 48^3x96 with 32 vectors, which does not
 * fit next to the setup's other fields on one GPU; the allocation then fails
 * with MRHS_ERR_OOM). MRHS_ERR_ARG unless even_odd is 0 or 1. */
int mrhs_set_smoother(mrhs_ctx ctx, int even_odd);

/* ------------------------------------------------------ setup building blocks */

/* copy ntv test vectors (device interleaved field, nrhs = ntv, storage
 * dtype) into the context's test-vector storage (converted to the context
 * precision's storage type) */
int mrhs_set_tv(mrhs_ctx ctx, const void* tv, int dtype);

/* P from the test vectors: per aggregate A and chirality h the vectors
 * v_1..v_ntv restricted to A x h are orthonormalised in order (Sec. 2: the
 * test vectors define P, and R is its adjoint); the result is the Q
 * factor of the thin QR with positive real diagonal, computed on the GPU
 * by two Cholesky-QR passes with double-precision Gram matrices.
 * MRHS_ERR_NONFINITE if a vector set is (numerically) dependent. */
int mrhs_build_P(mrhs_ctx ctx);

/* D_c = R D P (Sec. 2) as a 9-point stencil on the aggregate lattice:
 * Dc[A][k][2ntv][2ntv], k = 0 the aggregate itself, k = 1+mu the aggregate
 * A+mu, k = 5+mu the aggregate A-mu (the blocks are kept separate even when
 * A+mu == A-mu). MRHS_ERR_STATE before mrhs_build_P. */
int mrhs_build_Dc(mrhs_ctx ctx);

/* Engine of the contraction P^dag (D P) inside mrhs_build_Dc (the dense
 * 2ntv x 2ntv coarse-link products). AUTO: CUDA cores for FP64 contexts;
 * tensor cores (tcgen05, FP32 accumulation) otherwise: split tf32 for FP32
 * (as TC_TF32X3; the CUDA cores when 2*ntv > 64), bf16 operands for
 * MIX_BF16, tf32 for MIX_FP16. ALU:
 * always the CUDA cores. TC_BF16 / TC_F16 / TC_TF32: the tensor cores with
 * that operand type (P and D P rounded to it); TC_TF32X3: split tf32 (every
 * operand as hi + lo tf32 parts, products hi*hi + hi*lo + lo*hi, FP32
 * accuracy). The
 * tensor-core forms need FP32 work fields (prec FP32 or mixed) and
 * 2*ntv <= 64; mrhs_build_Dc returns MRHS_ERR_SHAPE otherwise,
 * MRHS_ERR_TIMEOUT if a bounded wait of the tensor-core pipeline ran out.
 * The backward blocks always follow from gamma_5-hermiticity. */
typedef enum {
  MRHS_DC_AUTO = 0,
  MRHS_DC_ALU = 1,
  MRHS_DC_TC_BF16 = 2,
  MRHS_DC_TC_F16 = 3,
  MRHS_DC_TC_TF32 = 4,
  MRHS_DC_TC_TF32X3 = 5
} mrhs_dc_engine;
int mrhs_set_dc_engine(mrhs_ctx ctx, int engine);

/* restriction vc = R v = P^dag v (Algorithm 3 of the paper, all nrhs at
 * once): vc[A][h*ntv+j] = sum_{x in A, c in h} conj(P_j(x,c)) v(x,c).
 * v: fine device field, vc: coarse device field, both of storage dtype
 * (F64 or F32; must match the context's compute type). */
int mrhs_restrict(mrhs_ctx ctx, const void* v, void* vc, int nrhs, int dtype);
/* prolongation u = P uc (Sec. 2, Algorithm 1) */
int mrhs_prolong(mrhs_ctx ctx, const void* uc, void* u, int nrhs, int dtype);
/* yc = D_c xc on nrhs coarse right-hand sides (Sec. 5: D_c applied with the
 * same broadcast scheme as the restriction). With F32 coarse fields, nrhs a
 * multiple of 16 up to 64, 2*ntv a multiple of 8 up to 64, an engine other
 * than MRHS_DC_ALU and pipeline stages that fit in shared memory (the split
 * form at 2*ntv = 64 takes up to 48 right-hand sides) the products run on the
 * tensor cores (tcgen05, FP32 accumulation): split tf32 (hi*hi + hi*lo +
 * lo*hi, FP32 accuracy) for FP32 contexts, single tf32 for the mixed ones;
 * otherwise on the CUDA cores. */
int mrhs_apply_Dc(mrhs_ctx ctx, const void* xc, void* yc, int nrhs, int dtype);

/* Approximate coarse solve of Algorithm 1/2 (relative tolerance 0.05 in Sec. 7):
 * GMRES(restart) on D_c xc = bc from xc = 0 for every right-hand side at
 * once, each with its own Krylov space; a right-hand side stops when its
 * residual estimate reaches tol*|bc| or after maxit iterations in total.
 * tol = 0 gives exactly maxit iterations. iters (host, may be NULL)
 * receives the iteration count of every right-hand side. With the even-odd
 * coarse solver (mrhs_set_coarse_solver) the GMRES runs on the Schur
 * complement instead and the tolerance applies to its right-hand side. */
int mrhs_coarse_solve(mrhs_ctx ctx, const void* bc, void* xc, int nrhs, int dtype, double tol, int restart,
                      int maxit, int* iters);

/* Coarse solver of every coarse solve (mrhs_coarse_solve, the refinement
 * phase, the V-cycle of mrhs_solve_fgmres). even_odd = 0 (default): GMRES on
 * D_c. even_odd = 1: even-odd preconditioning of the coarse system (Sec. 4,
 * Eq. 1): the aggregates take the red-black colour of their SAP domains, so
 * every hop block of D_c joins aggregates of different colour and D_ee, D_oo
 * are block diagonal (the self blocks); GMRES runs on
 *   S x_e = b_e - D_eo D_oo^-1 b_o,   S = D_ee - D_eo D_oo^-1 D_oe,
 * from x_e = 0 (the odd rows of the Krylov vectors stay zero), then
 * x_o = D_oo^-1 (b_o - D_oe x_e). The inverse self blocks of the odd
 * aggregates are built in the work precision on the first solve after each
 * build of D_c (MRHS_ERR_NONFINITE if one is singular, MRHS_ERR_SHAPE if a
 * 2ntv x 4ntv block does not fit in shared memory). The setting does not
 * apply to mrhs_coarse_solve_noalloc, which always solves on D_c.
 * MRHS_ERR_ARG unless even_odd is 0 or 1. */
int mrhs_set_coarse_solver(mrhs_ctx ctx, int even_odd);

/* The same coarse solve without any allocation. The paper has no counterpart:
 * this entry point is for callers that cannot let the library call
 * cudaMalloc (device memory handed out entirely by the caller's own pool or
 * caching allocator, no device-wide synchronisation wanted in the middle of
 * a solve, or no allocation allowed after start-up). The Krylov basis, the
 * GMRES state and the reduction partials live in one fixed 64 MiB device
 * array inside the library (held by every GPU that loads the library until
 * the process exits); results equal those of mrhs_coarse_solve with the
 * default coarse solver (GMRES on D_c, whatever mrhs_set_coarse_solver
 * says).
 * - MRHS_ERR_SHAPE (with the needed size in mrhs_last_error) when the
 *   problem needs more than 64 MiB: (restart + 2) coarse fields of nrhs
 *   right-hand sides plus the GMRES state and partials.
 * - The context's device must be the current device (MRHS_ERR_ARG if not).
 * - The first call on a device looks up the array's device address (this may
 *   load the library's device code on that device); make that first call
 *   before any stream capture.
 * - Every call uses the same array and leaves its contents behind; each
 *   call initialises everything it reads. Calls that overlap on the GPU
 *   (different streams or contexts at the same time) race on the array. */
int mrhs_coarse_solve_noalloc(mrhs_ctx ctx, const void* bc, void* xc, int nrhs, int dtype, double tol, int restart,
                              int maxit, int* iters);

/* ------------------------------------------------------------------ setup */

/* Initial phase (Sec. 2): the SAP smoother on every test vector from x0 = 0
 * (init_mode 0: one call of n_sweeps sweeps with b = v_j; init_mode 1:
 * n_sweeps calls of one sweep, each v_j <- SAP(b = v_j, x0 = 0)), each v_j
 * normalised, then P (mrhs_build_P) and D_c (mrhs_build_Dc). All test
 * vectors are processed at once. tv0: device interleaved field, nrhs = ntv,
 * storage dtype; read only, on the context's stream (with init_mode 0, one
 * block of all ntv vectors and dtype equal to the context's storage type,
 * the smoother reads it in place as its right-hand sides), so it must stay
 * valid and unchanged until the stream has passed the call. */
int mrhs_setup_init(mrhs_ctx ctx, const void* tv0, int dtype, int init_mode, int n_sweeps, int n_mr);

/* Iterative refinement, Algorithm 2 with block length N_b (default N_b =
 * ntv: all test vectors at once; see mrhs_set_block_length): n_iter times
 * { for each block of N_b test vectors in order: vc = R v; uc ~ D_c^-1 vc
 * (coarse GMRES, coarse_tol, coarse_restart, coarse_maxit); x = P uc;
 * x <- SAP^n_sweeps(b = v, x0 = x); v <- x normalised; after the last block
 * P and D_c rebuilt }.
 * coarse_iters (host, may be NULL): [n_iter][ntv] coarse iteration counts.
 * MRHS_ERR_STATE before mrhs_setup_init. */
int mrhs_setup_refine(mrhs_ctx ctx, int n_iter, int n_sweeps, int n_mr, double coarse_tol, int coarse_restart,
                      int coarse_maxit, int* coarse_iters);

/* Setup update after the gauge field has changed (the situation of HMC,
 * Sec. 1: the setup must be renewed every few solves): the caller has given
 * the new field (mrhs_set_gauge) and its clover term (mrhs_build_clover);
 * D_c is rebuilt from the kept P with the new operator, then n_iter
 * refinement iterations (as mrhs_setup_refine, same arguments) start from
 * the kept test vectors instead of new random ones. MRHS_ERR_STATE without an
 * earlier setup or before mrhs_build_clover. */
int mrhs_setup_update(mrhs_ctx ctx, int n_iter, int n_sweeps, int n_mr, double coarse_tol, int coarse_restart,
                      int coarse_maxit, int* coarse_iters);

/* Block length N_b of Algorithm 2 for mrhs_setup_init and
 * mrhs_setup_refine: the test vectors are processed in blocks of N_b in
 * order, the last block holding the remainder when N_b does not divide ntv
 * (the footnote to Algorithm 2). nb = 0 or nb >= ntv: all test vectors at
 * once (the default, N_b = N_tv). nb = 1 is the single-right-hand-side order
 * of Algorithm 1. Every N_b gives the same setup up to rounding (R, P and
 * D_c are fixed while the vectors are visited; only the order of the work
 * changes, Sec. 3); smaller blocks only take longer. MRHS_ERR_ARG if nb < 0.
 * The learned initial phase always takes all test vectors at once. */
int mrhs_set_block_length(mrhs_ctx ctx, int nb);

/* ------------------------------------------------- learned generator */

/* A gauge-covariant nearest-neighbour convolution network that maps test
 * vectors after one SAP sweep to near-null vectors (a project form beside the
 * paper's method; the paper itself has none). Channels are colour triplets;
 * widths = {4, C1, C2, 4}, C1, C2 <= 32 (a spinor is 4 spin channels x 3
 * colours). Layer: z(x)[c] = sum_{k=0..8} sum_c' W[k][c][c'] s_k T_k(x)
 * h(n_k(x))[c'] with k = 0 the site (T = 1), k = 1+mu the +mu neighbour
 * (T = U_mu(x)), k = 5+mu the -mu neighbour (T = U_mu(x-mu)^dag), s_k = -1 on
 * hops across the t boundary; modReLU h[c] = z[c] max(0,|z[c]|+b[c])/|z[c]|
 * after layers 1 and 2. Parameters (host float arrays): complex W of the three
 * layers ([9][C_out][C_in], (re, im) pairs) then the real biases b1[C1],
 * b2[C2]. bf16_weights != 0: forward and backward use the weights rounded to
 * bf16 (master copy and Adam state stay FP32). Fields are FP32 device fields
 * of the context. Gradients are dL/dRe + i dL/dIm. */
int mrhs_nn_create(mrhs_ctx ctx, const int widths[4], int bf16_weights);
int mrhs_nn_num_params(mrhs_ctx ctx, long long* n_complex, long long* n_real);
int mrhs_nn_set_weights(mrhs_ctx ctx, const float* host);
/* compute_copy != 0: the weights the kernels use (bf16-rounded if enabled) */
int mrhs_nn_get_weights(mrhs_ctx ctx, float* host, int compute_copy);
int mrhs_nn_get_grads(mrhs_ctx ctx, float* host);
int mrhs_nn_zero_grads(mrhs_ctx ctx);
/* out = net(in); keeps the activations for mrhs_nn_backward */
int mrhs_nn_forward(mrhs_ctx ctx, const void* in, void* out, int nrhs);
/* out = net(in) for inference (no activations kept; the right-hand sides in
 * chunks of at most 8). With bf16 weights the channel mixing of every layer
 * with 16 or more channels on one side runs on the tensor cores (tcgen05,
 * kind::f16): every transported input
 * triplet s_k T_k h(n_k) (the transport in FP32) is rounded once to bf16
 * (round to nearest even) when it enters the product, the weights are the
 * bf16 compute copy, products and sums are FP32; narrower layers and FP32
 * weights take the CUDA-core layer of mrhs_nn_forward. This is the network
 * mrhs_setup_init_learned applies. MRHS_ERR_TIMEOUT if a bounded wait of
 * the tensor-core pipeline ran out. */
int mrhs_nn_infer(mrhs_ctx ctx, const void* in, void* out, int nrhs);
/* accumulates the parameter gradients of a real loss with dL/dout given in
 * grad_out; grad_in (may be NULL) receives dL/din */
int mrhs_nn_backward(mrhs_ctx ctx, const void* grad_out, void* grad_in, int nrhs);
/* training loss L = sum_r |D v_r|^2/|v_r|^2 + lambda |v_r - P P^dag v_r|^2/|v_r|^2
 * with P the context's current prolongation (a plain setup of this gauge
 * field); grad_v (may be NULL) receives dL/dv; per_rhs (host, may be NULL)
 * the terms of every right-hand side */
int mrhs_nn_loss(mrhs_ctx ctx, const void* v, void* grad_v, int nrhs, double lambda, double* loss, double* per_rhs);
/* one Adam step (step counts from 1) on the accumulated gradients */
int mrhs_nn_adam(mrhs_ctx ctx, float lr, float beta1, float beta2, float eps, int step);
/* forward + loss + backward + Adam (beta 0.9, 0.999, eps 1e-8) on v_in */
int mrhs_nn_train_step(mrhs_ctx ctx, const void* v_in, int nrhs, double lambda, float lr, int step, double* loss);
/* learned initial phase: x = SAP^n_sweeps(b = tv0, x0 = 0), v = net(x)
 * normalised, then P and D_c (replaces the initial phase's SAP sweeps) */
int mrhs_setup_init_learned(mrhs_ctx ctx, const void* tv0, int dtype, int n_sweeps, int n_mr);

/* copy the test vectors / P out: host canonical [ntv][V][12] (complex128
 * for MRHS_F64, complex64 for MRHS_F32). Column j of P is the orthonormalised
 * v_j; its chirality-h part is the prolongation column (h, j). */
int mrhs_get_tv(mrhs_ctx ctx, void* host, int host_dtype);
int mrhs_get_P(mrhs_ctx ctx, void* host, int host_dtype);
/* copy D_c out: host [nagg][9][2ntv][2ntv] complex */
int mrhs_get_Dc(mrhs_ctx ctx, void* host, int host_dtype);

/* ------------------------------------------------- checkpoint / restore */

/* Write the finished setup to the file `path`: the test vectors, P and D_c,
 * the products of the setup phase (Sec. 2; Alg. 1/2) that later solves reuse.
 * The file holds a header (format version, lattice and aggregate extents,
 * ntv, precision, a hash of the device site order, the test-vector scale),
 * the three device images in the context's storage types, and a checksum.
 * The gauge field and the clover term are not in it. The file is first
 * written as `path`.part and renamed to `path` only once it is complete; on
 * failure the .part file is removed. MRHS_ERR_STATE before the setup has run
 * (no P or no D_c). MRHS_ERR_ARG when the file cannot be written. Waits for
 * the context's stream. */
int mrhs_save_setup(mrhs_ctx ctx, const char* path);
/* Replace the context's setup by the one in the file `path` (written by
 * mrhs_save_setup), bit for bit, so that mrhs_apply_Dc, the coarse solves,
 * mrhs_setup_refine and mrhs_solve_fgmres continue from it without a new
 * setup. The context must have the file's lattice and aggregate extents, ntv
 * and precision (MRHS_ERR_SHAPE otherwise). The gauge field and clover term
 * are the caller's to set, as for any setup, before anything that applies D.
 * MRHS_ERR_ARG for a file that cannot be opened, is not a checkpoint, is
 * truncated or fails its checksum; after a failure past the header checks
 * the context holds no setup (MRHS_ERR_STATE from calls that need one).
 * Waits for the context's stream. */
int mrhs_load_setup(mrhs_ctx ctx, const char* path);

/* ---------------------------------------------------------- measurement */

/* Per-kernel timing with CUDA events recorded on the context's stream around
 * every launch of the library's kernels. enable = 1 clears the counters and
 * starts recording; enable = 0 stops. Adds two event records per launch. */
int mrhs_profile(mrhs_ctx ctx, int enable);
/* Entry idx (0-based) of the per-kernel totals recorded so far (waits for
 * the stream): kernel class name (NUL-terminated, truncated to name_len),
 * number of launches and total milliseconds. MRHS_ERR_ARG past the last
 * entry. */
int mrhs_profile_read(mrhs_ctx ctx, int idx, char* name, int name_len, long long* launches, double* ms);

/* ------------------------------------------------ two-level FGMRES solve */

/* Two-level FGMRES(restart) on D x = b (Sec. 2: FGMRES preconditioned by the
 * multigrid V-cycle), outer Arnoldi, D and residual in FP64; the
 * preconditioner z = SAP^n_sweeps(b = r, x0 = P GMRES_c(R r)) runs in the
 * context precision. b, x: host canonical [V][12] complex128. Stops at
 * relative residual tol or maxit iterations. iters, relres: host, may be
 * NULL. MRHS_ERR_NOCONV when maxit is reached first (x is still written). */
int mrhs_solve_fgmres(mrhs_ctx ctx, const double* b, double* x, double tol, int restart, int maxit,
                      double coarse_tol, int coarse_restart, int coarse_maxit, int n_sweeps, int n_mr,
                      int* iters, double* relres);

#ifdef __cplusplus
}
#endif

#endif /* MRHS_H */
