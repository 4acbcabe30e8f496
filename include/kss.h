/*
 * kss.h -- C ABI of the GB300 plane-wave Kohn-Sham Hamiltonian / Chebyshev-filter library.
 *
 * What is computed (arXiv 2507.08578):
 *   The Kohn-Sham eigenproblem in a plane-wave basis, Hartree atomic units (§1), with
 *     H = -1/2 nabla^2 + V_loc + sum_i |beta_i> D_i <beta_i|
 *   the separable nonlocal operator of the nonlocal-Hamiltonian equation (Eq. ham-nl, §5.2) with
 *   the diagonal h of norm-conserving pseudopotentials, the projector table and the projector
 *   coefficients ("cprj") kept in memory so that every nonlocal step is a matrix product (§5.2),
 *   the local part applied by batched FFTs over bands (§5.1), and the lowest bands found by a
 *   Chebyshev-filtered subspace iteration with Rayleigh-Ritz (§5.1).
 *
 * Conventions shared by every entry point:
 *   - All functions return kss_status.  No C++ exception crosses this boundary.  On failure a
 *     message is stored in the context (kss_last_error) and outputs are left unspecified.
 *   - Wavefunction blocks are band-major: band n of a block occupies elements
 *     [n*ld, n*ld + npw) of an array of complex numbers; ld >= npw.  Complex numbers are
 *     interleaved (re, im) pairs: complex128 (2 x double) for KSS_PREC_FP64, complex64
 *     (2 x float) for KSS_PREC_MIXED.
 *   - Plane-wave order (the "G-sphere"): Miller triples m with 0.5*|k+G|^2 <= ecut, where
 *     k+G = sum_i (m_i + kappa_i) b_i, sorted ascending by (m3, m2, m1), m1 fastest.
 *   - Device pointers are CUDA device (or managed) addresses on the context's device; the
 *     caller owns them and keeps them alive until the work queued on the context stream that
 *     uses them has finished.  Host pointers are ordinary host memory.
 *   - All GPU work is queued on the context stream (stream-ordered); calls that return host
 *     results synchronise that stream before returning.
 *   - A context is not thread-safe: one host thread at a time per context.
 *   - There is no CPU fallback: without a usable CUDA device kss_create fails with KSS_ECUDA.
 */
#ifndef KSS_H
#define KSS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define KSS_VERSION_MAJOR 0
#define KSS_VERSION_MINOR 1

typedef enum {
  KSS_OK = 0,
  KSS_EINVAL = 1,    /* bad argument (null pointer, size out of range, inconsistent sizes) */
  KSS_ENOMEM = 2,    /* device or host allocation failed */
  KSS_ECUDA = 3,     /* CUDA / cuSOLVER error, or no usable device */
  KSS_ENOCONV = 4,   /* eigensolver hit max_iter; outputs hold the last iterate */
  KSS_ETIMEOUT = 5,  /* a bounded device-side wait gave up */
  KSS_EBUSY = 6,     /* admission refused (memory budget or slot limit) */
  KSS_ENUMERIC = 7,  /* non-finite values or a failed factorisation */
  KSS_ENOTSUP = 8    /* valid request this build does not support */
} kss_status;

typedef enum { KSS_PREC_FP64 = 0, KSS_PREC_MIXED = 1 } kss_precision;

typedef struct kss_ctx_s* kss_ctx;
typedef struct kss_sys_s* kss_sys;
typedef struct kss_solver_s* kss_solver;

/* ------------------------------------------------------------------------------------------
 * Context (device and stream plumbing; no counterpart in the paper)
 * ------------------------------------------------------------------------------------------ */

/* Create a context on CUDA device `device` that queues all its work on `cuda_stream`, a
 * cudaStream_t of that device (borrowed: it must outlive the context).  NULL is the CUDA legacy
 * default stream (stream 0), the stream PyTorch uses unless told otherwise, so work queued by
 * the caller on that stream and by the library is ordered.
 * Errors: KSS_EINVAL (out == NULL), KSS_ECUDA (no device / bad device index). */
kss_status kss_create(kss_ctx* out, int device, void* cuda_stream);

/* Destroy a context.  Every system created on it must be destroyed first (KSS_EINVAL otherwise).
 * Synchronises the stream. */
kss_status kss_destroy(kss_ctx ctx);

/* Message of the last failed call on this context ("" if none).  Owned by the context; valid
 * until the next call on it.  Cannot fail: accepts NULL (returns a static message). */
const char* kss_last_error(kss_ctx ctx);

/* Library version as major*1000 + minor (no counterpart in the paper).  Cannot fail. */
int kss_version(void);

/* ------------------------------------------------------------------------------------------
 * Systems: cell, cutoff, k-points, atoms (setup, §1 / §5.2)
 * ------------------------------------------------------------------------------------------ */

typedef struct {
  double lattice[9];       /* rows a1, a2, a3 (bohr), row-major */
  double ecut;             /* plane-wave cutoff (Ha), > 0 */
  int nk;                  /* number of k-points, >= 1 */
  const double* kpts_red;  /* host, nk*3 reduced coordinates (copied at setup) */
  int fft_box[3];          /* FFT grid N1,N2,N3; all 0 => smallest {2,3,5}-smooth N_i >= 4 max|m_i|+1 */
} kss_cell;

typedef struct {
  int natom;               /* >= 0 */
  const double* pos_cart;  /* host, natom*3 Cartesian positions (bohr), copied */
  double vloc_amp;         /* A of V(r) = A sum_a sum_L exp(-|r-R_a-L|^2/(2 sigma^2)) (Ha) */
  double vloc_sigma;       /* sigma (bohr), > 0 */
  int nproj_per_atom;      /* 0, 1 (s) or 4 (s, px, py, pz) */
  double proj_alpha;       /* form factor exp(-alpha |k+G|^2), > 0 */
  const double* D;         /* host, natom*nproj_per_atom projector energies (Ha), copied;
                              index 4a+l for l in (s, px, py, pz) */
  const double* Q;         /* host, natom*nproj_per_atom overlap coefficients q_i (same index),
                              copied, or NULL.  With Q the eigenproblem is the generalised
                              H psi = lambda S psi, S = 1 + sum_i |beta_i> q_i <beta_i| (§5.2:
                              the nonlocal part of the overlap has the structure of Eq. ham-nl);
                              S must be provably positive definite: 1 + min(0, min q) * g > 0,
                              g the Gershgorin bound of the largest eigenvalue of the projector
                              Gram matrix beta^H beta (KSS_EINVAL otherwise).  NULL or all-zero
                              Q: S = 1, the standard problem. */
} kss_atoms;

/* Build a system: enumerate the G-sphere of every k-point on the host (the inclusion test is
 * evaluated in IEEE double without contraction, exactly as written in the convention above),
 * upload the index maps, and fill on the device the local potential on the FFT grid (full
 * periodic-image sum of the Gaussians; terms below 1e-20*|A| omitted), the kinetic energies
 * 0.5|k+G|^2 and the projector table beta_{a,l}(k+G) = c_l q_l exp(-alpha|q|^2) exp(-i q.R_a)
 * (q_s = 1; c_s, c_p the continuum unit-norm constants).  Library-owned device memory.
 * Errors: KSS_EINVAL (bad cell/atoms, FFT box too small for the sphere or not {2,3,5}-smooth,
 * box dimension > 256), KSS_ENOMEM, KSS_ECUDA. */
kss_status kss_setup(kss_ctx ctx, const kss_cell* cell, const kss_atoms* atoms, kss_sys* out);

/* Waits for the context's stream and frees the system's device tables.  Errors: KSS_EINVAL
 * (NULL, or solvers of this system still alive: destroy them first; the system is kept). */
kss_status kss_sys_destroy(kss_sys sys);

typedef struct {
  int nk;
  int fft_box[3];
  int nproj;
  int npw_max;
  double volume;           /* bohr^3 */
  double vloc_max;         /* max_j V(r_j) */
} kss_sys_info;

/* Sizes of a system as set up (host struct filled by the call).  Errors: KSS_EINVAL (NULL). */
kss_status kss_sys_info_get(kss_sys sys, kss_sys_info* out);

/* Number of plane waves of k-point ik and a library-owned host copy of its Miller triples
 * (npw*3 int32, canonical order; the plane-wave basis of §1 and §5.2), valid until the system is
 * destroyed; miller_host may be NULL.  Errors: KSS_EINVAL (NULL sys/npw, ik out of range). */
kss_status kss_sphere(kss_sys sys, int ik, int* npw, const int32_t** miller_host);

/* Host-only queries: no context and no device needed (the same host code kss_setup runs).
 * kss_sphere_host: the G-sphere of one k-point, {m : 0.5|k+G_m|^2 <= ecut} in the canonical
 * order of kss_sphere (ascending m3, m2, m1; the inclusion test evaluated in IEEE double without
 * contraction, §1 and §5.2 plane-wave basis).  lattice: 9 doubles, rows a1, a2, a3 in bohr;
 * kred: 3 reduced coordinates.  *npw receives the count; miller (host, caller-owned, may be NULL
 * to query the count) receives npw triples when cap >= npw.  Errors: KSS_EINVAL (null npw/kred,
 * non-finite or singular lattice, ecut <= 0, cap < npw with miller given), KSS_ENOMEM.
 * kss_default_box: the FFT box kss_setup uses when the cell gives none: per axis the smallest
 * {2,3,5}-smooth N_i >= 4 max|m_i| + 1 over the spheres of all nk k-points (kpts_red: nk * 3).
 * Errors: KSS_EINVAL, KSS_ENOMEM (these two calls have no context, so no message is stored). */
kss_status kss_sphere_host(const double* lattice, double ecut, const double* kred, int cap, int* npw,
                           int32_t* miller);
kss_status kss_default_box(const double* lattice, double ecut, int nk, const double* kpts_red, int* box);

/* Copy back from DEVICE memory the index maps the kernels use: miller (npw*3 int32) and the box
 * offsets (m1 mod N1) + N1*((m2 mod N2) + N2*(m3 mod N3)) (npw int32), into caller-owned host
 * buffers (either may be NULL); synchronises the context's stream first.  Errors: KSS_EINVAL
 * (ik out of range), KSS_ECUDA. */
kss_status kss_get_maps(kss_sys sys, int ik, int32_t* miller_out, int32_t* offset_out);

/* Copy back from device the local potential V(r_j) (N1*N2*N3 doubles, index j1 + N1*(j2 +
 * N2*j3), not scaled), the kinetic energies 0.5|k+G|^2 (npw doubles) and the projector table of
 * Eq. ham-nl (§5.2) (npw*nproj complex128, projector-major: element (i, g) at [i*npw + g]) into
 * caller-owned host buffers.  Any output may be NULL; synchronises the context's stream first.
 * Errors: KSS_EINVAL (ik out of range), KSS_ECUDA. */
kss_status kss_get_tables(kss_sys sys, int ik, double* vloc_out, double* kinetic_out,
                          double* beta_out);

/* Rigorous upper bound of the spectrum of H(k): max T + max(max V, 0) + sum_i max(D_i,0)|beta_i|^2
 * (the upper end of the Chebyshev filter interval, §5.1; for a system with an overlap the bound of
 * S^-1 H).  Errors: KSS_EINVAL (NULL, ik out of range). */
kss_status kss_upper_bound(kss_sys sys, int ik, double* bound);

/* Device bytes the solver needs for nband bands at this precision (all k-points handled one at
 * a time), excluding the system tables already allocated (no counterpart in the paper; used for
 * admission by memory footprint).  Errors: KSS_EINVAL (NULL, nband < 1). */
kss_status kss_footprint(kss_sys sys, int nband, kss_precision prec, size_t* bytes);

/* ------------------------------------------------------------------------------------------
 * Hamiltonian application on a band block (§5.1 batched FFTs; §5.2 Eq. ham-nl)
 * ------------------------------------------------------------------------------------------ */

/* hpsi = H(k_ik) psi for nb bands.  psi, hpsi: DEVICE, band-major [nb][ld], complex128 for
 * KSS_PREC_FP64 and complex64 for KSS_PREC_MIXED; they must not overlap.  Steps: projector
 * coefficients C = beta^H psi; per band, sphere -> box scatter, inverse 3D FFT, x V(r), forward
 * 3D FFT, box -> sphere gather, + 0.5|k+G|^2 psi; then hpsi += beta (D C).
 * nb == 0 is a no-op.  Errors: KSS_EINVAL (ik out of range, nb < 0, ld < npw, null pointers).
 * The call is stream-ordered and does not synchronise: if a bounded wait inside a
 * KSS_PREC_MIXED projector product gave up, the next call of this context that synchronises
 * (a solver step or solve, kss_gemm) returns KSS_ETIMEOUT. */
kss_status kss_apply_H(kss_sys sys, int ik, int nb, const void* psi, void* hpsi, int ld,
                       kss_precision prec);

/* kss_apply_H for real-space-real bands at k = 0 (psi(-G) = conj psi(G) for every band, the
 * caller's guarantee): two bands per complex FFT (psi_a + i psi_b), then
 * H psi_a = T psi_a + (F(G) + conj F(-G))/2 + nonlocal, H psi_b = T psi_b + (F(G) - conj F(-G))/2i
 * + nonlocal, F the transform of V (psi_a + i psi_b) (the time-reversal economy the paper notes for
 * Gamma, §6).  Same arguments as kss_apply_H; KSS_EINVAL if k-point ik is not Gamma. */
kss_status kss_apply_H_gamma(kss_sys sys, int ik, int nb, const void* psi, void* hpsi, int ld,
                             kss_precision prec);

/* spsi = S(k_ik) psi = psi + beta (Q (beta^H psi)): the overlap of a system set up with Q
 * (spsi = psi without it; §5.2, the nonlocal overlap with the structure of Eq. ham-nl).  Same
 * layout and rules as kss_apply_H.  Errors: KSS_EINVAL (ik out of range, nb < 0, ld < npw, unknown
 * precision, null or identical psi / spsi). */
kss_status kss_apply_S(kss_sys sys, int ik, int nb, const void* psi, void* spsi, int ld,
                       kss_precision prec);

/* One Chebyshev three-term step (the filter of the Chebyshev-filtered subspace iteration, §5.1)
 * fused into the application of the filter operator F:
 *   out = alpha * F psi + beta * psi + gamma * psi_prev
 * F = H, or F = S^-1 H for a system with an overlap (S^-1 = 1 - beta W beta^H with the
 * precomputed W = Q (1 + beta^H beta Q)^-1 per k-point).
 * psi_prev may be NULL (then gamma is ignored) and may alias out (out is written element by
 * element after psi_prev at the same element is read).  psi must not overlap out.  Layout and
 * stream ordering as kss_apply_H.  Errors: as kss_apply_H. */
kss_status kss_cheb_step(kss_sys sys, int ik, int nb, const void* psi, const void* psi_prev,
                         void* out, int ld, double alpha, double beta, double gamma,
                         kss_precision prec);

/* kss_apply_H with HOST psi/hpsi (caller-owned, band-major [nb][ld]; pinned memory makes the
 * copies asynchronous): copies psi to library-owned device staging, applies H and copies the
 * result back; synchronises the stream before returning.  Errors: KSS_EINVAL (ik out of range,
 * nb < 0, ld < npw, null buffers), KSS_ENOMEM, KSS_ECUDA. */
kss_status kss_apply_H_host(kss_sys sys, int ik, int nb, const void* psi_host, void* hpsi_host,
                            int ld, kss_precision prec);

/* Size of the static device scratch array used by kss_apply_H_noalloc (64 MiB). */
#define KSS_NOALLOC_SCRATCH_BYTES (64u * 1024u * 1024u)

/* kss_apply_H for callers that cannot allocate device memory.  The paper has no counterpart:
 * this is a deployment variant of the H application above.
 *
 * Who needs it: code that must not call cudaMalloc/cudaFree at this point -- work recorded
 * while a CUDA stream is being captured into a graph, a host whose device memory belongs to
 * another allocator (a framework's caching allocator or a fixed-budget pool), or a latency-
 * critical loop where an allocation and the device-wide synchronisation of cudaFree are not
 * acceptable.  kss_apply_H may grow the context's workspaces; this call never allocates: it
 * calls no cudaMalloc, cudaFree or allocating library routine.
 *
 * Same arguments, layout and result as kss_apply_H (psi, hpsi: caller-owned DEVICE band blocks
 * [nb][ld]).  Every temporary (the FFT slab of a band chunk, the projector coefficients, the
 * split-K partial sums) lives in one file-scope device array of KSS_NOALLOC_SCRATCH_BYTES that
 * every GPU which loads the library holds until the process exits.  The nonlocal products run
 * on the CUDA cores in both precisions (the tensor-core path needs operand buffers larger than
 * the scratch), so MIXED results agree with kss_apply_H to single-precision rounding.
 *
 * The first call on each context looks up the array's device address (cudaGetSymbolAddress,
 * with the context's device current) and keeps it in the context; make that first call before
 * any stream capture.  With CUDA's default lazy module loading, the first call in a process on a
 * device is also when the device commits the array's KSS_NOALLOC_SCRATCH_BYTES (the module that
 * holds it is loaded then); every later call, on any context of that device, commits nothing.
 * All calls share the array and it keeps the last call's contents; nothing in it needs to start
 * at zero (every byte read is written first by the same call).  Calls whose work overlaps on
 * the GPU (two streams, or two contexts on one device) race on the array: order them.
 * Errors: as kss_apply_H, plus KSS_EINVAL with a message when one band's FFT slab plus the
 * projector coefficients and one set of partial sums exceed KSS_NOALLOC_SCRATCH_BYTES (split
 * the band block).  Launches are not counted by kss_profile_*. */
kss_status kss_apply_H_noalloc(kss_sys sys, int ik, int nb, const void* psi, void* hpsi, int ld,
                               kss_precision prec);

/* Complex GEMM of the path (projector products, Eq. ham-nl of §5.2; Gram / projected-H /
 * rotation products of Rayleigh-Ritz, §5.1), exposed for direct testing and reuse.
 *   op 0: C = alpha A^H B + beta C, A is K x M (lda >= K), B is K x N (ldb >= K)
 *   op 1: C = alpha A B + beta C,   A is M x K (lda >= M), B is K x N (ldb >= K)
 * Column-major DEVICE matrices; C is M x N (ldc >= M) and must not overlap A or B.
 * KSS_PREC_FP64: complex128 on the FP64 pipe.  KSS_PREC_MIXED: complex64 on the tensor cores,
 * every FP32 value split into BF16 hi + lo, products hi*hi + hi*lo + lo*hi accumulated in FP32
 * (relative error of order 1e-5).  Errors: KSS_EINVAL, KSS_ETIMEOUT (a bounded device wait gave
 * up; the context stays usable). */
kss_status kss_gemm(kss_ctx ctx, int op, int M, int N, int K, const void* A, int lda, const void* B,
                    int ldb, void* C, int ldc, double alpha_re, double alpha_im, double beta_re,
                    double beta_im, kss_precision prec);

/* Dense FP64 generalised Hermitian eigensolve A x = lambda B x, the subspace problem of
 * Rayleigh-Ritz (§5.1: the projected H and the Gram matrix of the filtered block; Cholesky
 * orthonormalisation and the Rayleigh-Ritz eigensolve in one), exposed for direct testing and
 * reuse.  count independent pencils: pencil i has order n[i] >= 0 and DEVICE complex128
 * column-major matrices A[i] (lda[i] >= max(1, n[i])) and B[i] (ldb[i] >= max(1, n[i])), of
 * which only the lower triangles are read; B[i] must be Hermitian positive definite.  On return
 * the leading n x n block of A[i] holds the eigenvectors (columns, B-orthonormal, eigenvalues
 * ascending), w[i] (DEVICE, n[i] doubles) the eigenvalues, B[i] its Cholesky factor (lower) and
 * info[i] (HOST) 0, or j + 1 when B[i] is not positive definite at column j (outputs then
 * undefined).  real != 0: the pencils are real symmetric (imaginary parts ignored; solved in
 * real arithmetic; eigenvectors and factor written with zero imaginary parts).  Hand-written
 * kernels (Cholesky, reduction to standard form, Householder tridiagonalisation, bisection and
 * inverse iteration, back-transformation): one CTA per pencil, or a cooperative grid for a
 * single pencil of order >= 32.  Synchronises the context stream.
 * Errors: KSS_EINVAL (count < 0, NULL arrays, bad sizes), KSS_ETIMEOUT (a bounded grid-barrier
 * wait gave up), KSS_ECUDA. */
kss_status kss_dense_hegv(kss_ctx ctx, int count, const int* n, void* const* A, const int* lda,
                          void* const* B, const int* ldb, double* const* w, int* info, int real);

/* Phase times of the last single-pencil solve that ran on a cooperative grid (order >= 32) in
 * this context, from the device clock: ms[0] Cholesky (with the real-pencil input copy), ms[1]
 * reduction to standard form, ms[2] tridiagonalisation, ms[3] eigenvalues of the tridiagonal
 * matrix (bisection), ms[4] its eigenvectors (inverse iteration), ms[5] back-transformation.  Measurement support (the paper has no counterpart).  Synchronises the context stream; all zeros when
 * no grid solve has completed.  Errors: KSS_EINVAL (NULL), KSS_ECUDA. */
kss_status kss_dense_hegv_phase_ms(kss_ctx ctx, double* ms);

/* Failure path of the bounded device waits, exercised without a fault (test support; the paper
 * has no counterpart).  Launches one thread that waits on a device word nothing writes, with the
 * same %globaltimer limit pattern as the tensor-core pipeline waits; after limit_ms (0 < limit_ms
 * <= 1000) it gives up and raises the context's device error flag, which this call reads back.
 * Returns KSS_ETIMEOUT (the expected outcome) with the flag cleared and the context usable;
 * KSS_EINVAL for a limit out of range. */
kss_status kss_selftest_bounded_wait(kss_ctx ctx, double limit_ms);

/* Measured fused multiply-add throughput of the CUDA cores on the context's device, the
 * denominator of the ALU rooflines of the FFT passes (measurement support; the paper has no
 * counterpart).  pipe 0: FP64, 1: FP32.  Every thread of a grid of 8 CTAs per SM runs 8
 * independent FMA chains; *tflops is the best of three timed launches (2 flops per FMA, CUDA
 * events on the context stream; synchronises it).  Errors: KSS_EINVAL (NULL, pipe not 0 or 1),
 * KSS_ECUDA. */
kss_status kss_peak_probe(kss_ctx ctx, int pipe, double* tflops);

/* ------------------------------------------------------------------------------------------
 * Electron density after the solve (Eq. nandtau, §2)
 * ------------------------------------------------------------------------------------------ */

/* rho[j] += sum_n occ[n] |psi_n(r_j)|^2 on the FFT grid, with psi_n(r) = Omega^-1/2 sum_G
 * psi_n(G) e^{i(k+G).r} and r_j = sum_i (j_i/N_i) a_i.  psi: DEVICE band-major [nb][ld] of the
 * precision's type; occ: HOST, nb weights (occupancy times k-point weight; copied); rho: DEVICE
 * real double [N3][N2][N1] (j1 fastest), accumulated, so a caller sums k-points by calling once
 * per k-point on a zeroed rho.  Inverse FFTs per band (sphere scatter + x, y, z transforms) in the
 * precision's arithmetic, |psi|^2 accumulated in FP64 in a fixed order (bitwise reproducible).
 * Errors: KSS_EINVAL (ik, nb, ld, null pointers, non-finite occ), KSS_ENOTSUP (boxes with
 * N2 != N3 or a length without a two-codelet split). */
kss_status kss_density_accumulate(kss_sys sys, int ik, int nb, const void* psi, int ld,
                                  const double* occ, double* rho, kss_precision prec);

/* ------------------------------------------------------------------------------------------
 * Chebyshev-filtered subspace iteration with Rayleigh-Ritz (§5.1)
 * ------------------------------------------------------------------------------------------ */

typedef struct {
  int degree;              /* filter polynomial degree m (>= 1; 0 => 10) */
  double tol;              /* residual tolerance |H x - lambda S x| (Ha) on the wanted bands (<= 0 => 1e-8
                              in FP64; in the mixed form max(1e-5, 2e-6 x the spectral upper bound),
                              twice the single-precision floor of the residual) */
  int max_iter;            /* filter iterations (<= 0 => 200) */
  int nbuffer;             /* extra bands (< 0 => max(4, ceil(nband/10))) */
  kss_precision prec;
  uint64_t seed;           /* initial block: Philox4x32-10 uniform(-1,1) re/im from this seed */
  const void* x0;          /* optional DEVICE warm start, band-major [nb_x0][x0_ld], prec type */
  int x0_nb;               /* bands in x0 (<= nband+nbuffer; the rest are random) */
  int x0_ld;
  int flags;               /* KSS_SOLVE_* bits, 0 for the defaults */
} kss_solve_opts;

/* At k = 0 (Gamma) the solvers keep the bands real in real space, psi(-G) = conj psi(G) (the
 * start block and warm starts are symmetrised, Rayleigh-Ritz rotations are real), and the
 * ChebFi filter packs two bands per complex FFT (psi_a + i psi_b), halving the FFT work (the
 * time-reversal economy the paper notes for Gamma, §6).  This flag turns that off. */
#define KSS_SOLVE_NO_GAMMA_REAL 1
/* kss_solve_batch and the server: issue the filter's grouped launches directly instead of replaying
 * them as a CUDA graph (same results; every launch is then timed by kss_profile_*, which sees a
 * replayed graph as one entry). */
#define KSS_SOLVE_BATCH_NO_GRAPH 2
/* kss_solve_batch and the server, mixed form: the projector products of the batch on the FP32 CUDA
 * cores (FP32 accumulation) instead of the split-BF16 tensor-core products. */
#define KSS_SOLVE_BATCH_FP32_PROJ 4

typedef struct {
  int iters;               /* filter iterations done */
  long long napply;        /* band H-applications done (bands x applications) */
  double max_resid;        /* max residual over the wanted bands, last iterate (Ha) */
  double ms_filter, ms_rr, ms_total;
  int nb;                  /* block size nband + nbuffer actually used */
} kss_solve_stats;

/* Solver objects allow stepping one iteration at a time (used by the batched and served
 * paths).  create: allocates the block buffers and draws / copies the initial block.
 * Errors: KSS_EINVAL (nband < 1, nband+nbuffer > npw), KSS_ENOMEM. */
kss_status kss_solver_create(kss_sys sys, int ik, int nband, const kss_solve_opts* opts,
                             kss_solver* out);
/* Waits for the context's stream and frees the solver's blocks.  Errors: KSS_EINVAL (NULL). */
kss_status kss_solver_destroy(kss_solver s);

/* One iteration.  The first call performs the initial Rayleigh-Ritz on the starting block; each
 * later call filters (degree m), then Rayleigh-Ritz (FP64 Cholesky of the Gram matrix and FP64
 * Hermitian eigensolve on the GPU), then residuals.  *converged is set to 1 when every wanted
 * band has residual <= tol.  Synchronises the stream (the residuals decide convergence).
 * Errors: KSS_EINVAL (NULL), KSS_ENUMERIC (a failed factorisation or a non-finite Ritz value or
 * residual), KSS_ETIMEOUT (a bounded device wait of a mixed-precision projector product gave
 * up), KSS_ENOMEM, KSS_ECUDA; after an error the iterate is undefined. */
kss_status kss_solver_step(kss_solver s, int* converged);

/* One iteration on each of n solvers of the same context (e.g. the k-points of one system; §5.3
 * notes that k-points are independent), with the same results as n calls of kss_solver_step in
 * order.  The Rayleigh-Ritz of solver i (Gram products, the FP64 generalised eigensolve, the
 * rotations and residuals, §5.1) runs on a helper stream of the context while the filter of
 * solver i+1 runs on the context stream: the dense eigensolve is latency-bound and would
 * otherwise leave the GPU mostly idle.  Solvers that have not taken their first step do it
 * (initial Rayleigh-Ritz) in order first; solvers that are done are skipped, and a solver listed
 * twice steps once.  converged: NULL or an int array [n] set like kss_solver_step's flag.
 * Errors: KSS_EINVAL (n < 0, a NULL solver, solvers of different contexts), and those of
 * kss_solver_step; as after a failed kss_solver_step, the iterates are then undefined (the
 * filter works in place) and the solvers should be destroyed.  The stepped solvers' ms_filter
 * and ms_rr receive equal shares of the call's wall time. */
kss_status kss_solver_step_many(int n, kss_solver const* solvers, int* converged);

/* Results of the current iterate (the Ritz pairs of the last Rayleigh-Ritz, §5.1): evals/resid
 * host [nband] (may be NULL); evecs DEVICE band-major [nband][ld] of the solver's precision or
 * NULL; stats may be NULL.  Errors: KSS_EINVAL (NULL, no step taken yet, ld < npw), KSS_ECUDA. */
kss_status kss_solver_results(kss_solver s, double* evals, double* resid, void* evecs, int ld,
                              kss_solve_stats* stats);

/* Full solve = create + step until converged or max_iter + results + destroy (ChebFi with
 * Rayleigh-Ritz, §5.1).  evals/resid: host [nband] (may be NULL); evecs: DEVICE band-major
 * [nband][ld] of the precision's type, or NULL.  Returns KSS_ENOCONV (outputs still filled) when
 * max_iter is reached; other errors as kss_solver_create and kss_solver_step.
 * For a system with an overlap (kss_atoms.Q) the solver returns the lowest generalised
 * eigenpairs H x = lambda S x: the filter polynomial is in S^-1 H, Rayleigh-Ritz uses the
 * metric Y^H S Y, residuals are |H x - lambda S x|, and the eigenvectors are S-orthonormal. */
kss_status kss_chebfi_solve(kss_sys sys, int ik, int nband, const kss_solve_opts* opts,
                            double* evals, void* evecs, int ld, double* resid,
                            kss_solve_stats* stats);

/* LOBPCG, the paper's second GPU eigensolver (§5.1): the lowest nband eigenpairs with the
 * locally optimal block preconditioned conjugate gradient on one block of nband + nbuffer bands
 * (Teter-Payne-Allan preconditioner; H applied to the preconditioned residuals only, H X and H P
 * carried by linear combination; Rayleigh-Ritz in [X W P] by an FP64 generalised eigensolve).
 * Same arguments and outputs as kss_chebfi_solve (opts.degree ignored; max_iter <= 0 => 500).
 * FP64 only.  Errors: KSS_ENOTSUP (mixed precision, a system with an overlap), KSS_EINVAL
 * (3 (nband + nbuffer) > npw), KSS_ENOCONV (outputs still filled), KSS_ENUMERIC. */
kss_status kss_lobpcg_solve(kss_sys sys, int ik, int nband, const kss_solve_opts* opts,
                            double* evals, void* evecs, int ld, double* resid,
                            kss_solve_stats* stats);

/* RMM-DIIS refinement (§5.1: residual minimisation with direct inversion in the iterative
 * subspace, Kresse & Furthmueller): from trial vectors (opts->x0, at least nband bands; the rest
 * of the nband + nbuffer block is random), repeated sweeps of three per-band steps
 * psi_(j+1) = psibar_j + lambda K R(psibar_j), psibar_j the combination of the band's trials with
 * least residual norm (coefficients summing to one), lambda the optimal step of the first step, K
 * the Teter-Payne-Allan preconditioner, followed by one Rayleigh-Ritz (a single Cholesky
 * orthonormalisation) per sweep.  It converges to the eigenvectors nearest the trial vectors, so
 * the trial block must already resolve the wanted states (e.g. a solve at a loose tolerance or a
 * nearby system), and should cover the whole block (x0_nb = nband + nbuffer): random buffer bands
 * slow the convergence of the top of the window to a crawl.  Same outputs as kss_chebfi_solve (stats.iters = sweeps; max_iter <= 0 => 100).
 * FP64 only.  Errors: KSS_EINVAL (no x0 or x0_nb < nband), KSS_ENOTSUP (mixed precision, an
 * overlap), KSS_ENOCONV (outputs still filled), KSS_ENUMERIC. */
kss_status kss_rmmdiis_solve(kss_sys sys, int ik, int nband, const kss_solve_opts* opts,
                             double* evals, void* evecs, int ld, double* resid,
                             kss_solve_stats* stats);

/* ------------------------------------------------------------------------------------------
 * Batched solves: many systems / k-points in lockstep (§5.1 batch processing)
 * ------------------------------------------------------------------------------------------ */

/* Solve n independent (system, k-point) units of uneven sizes together: every iteration issues
 * the FFT passes of all units as single grouped launches and the projector products as grouped
 * GEMMs, the whole filter (degree m + the H application on the filtered block) being one CUDA
 * graph captured once and replayed with new coefficients; Rayleigh-Ritz (FP64 eigensolve) runs
 * per unit with one host synchronisation per iteration.  Units stop when converged.
 * sys[u] (same context), ik[u], nband[u]; opts is shared (precision, degree, tol, max_iter,
 * nbuffer; unit u draws its start block with seed opts->seed + u; x0 must be NULL).
 * evals[u], resid[u]: host arrays of nband[u] (any pointer may be NULL); stats: array of n or
 * NULL.  Returns KSS_ENOCONV if any unit hit max_iter (results still filled); KSS_ENOTSUP if a
 * unit's FFT lengths have no two-codelet split (125, 162, 200, 216, 243, 250) or its system has
 * an overlap (generalised problems are solved per system). */
kss_status kss_solve_batch(kss_ctx ctx, int n, const kss_sys* sys, const int* ik, const int* nband,
                           const kss_solve_opts* opts, double* const* evals, double* const* resid,
                           kss_solve_stats* stats);

/* ------------------------------------------------------------------------------------------
 * Request server: continuous batching of eigensolves as they arrive (the high-throughput
 * campaigns of many independent calculations, §7; the serving loop itself has no counterpart)
 * ------------------------------------------------------------------------------------------ */

typedef struct {
  long long completed, rejected, warm_hits;
  double p50_ms, p99_ms, mean_ms;  /* latency submit -> done, over completed requests */
  double solves_per_s;             /* completed requests / (last completion - first submit) */
  size_t peak_bytes, in_flight_bytes;  /* admission accounting: device bytes of the admitted requests
                                        (system tables + one solver footprint per k-point) */
} kss_server_stats;

/* Start a server on the context.  Requests are admitted in arrival order while the sum of their
 * estimated device footprints stays within hbm_budget_bytes and their k-points fit in max_slots
 * units; each admitted request's system tables and solver blocks stay resident until it
 * completes.  opts (shared by all requests; x0 must be NULL): precision, degree, tol, max_iter,
 * nbuffer, seed.  A warm-start cache of up to a tenth of the budget keeps the converged
 * subspace of finished requests; a later request with identical content starts from it.
 * While the server runs, the context belongs to it: other calls on the context are not allowed
 * until kss_server_stop. */
/* Errors: KSS_EINVAL (NULL, a server already running, zero budget or slots, opts with x0,
 * unknown precision). */
kss_status kss_server_start(kss_ctx ctx, size_t hbm_budget_bytes, int max_slots,
                            const kss_solve_opts* opts);

/* Queue a request (cell, atoms, nband: copied).  *ticket identifies it.  KSS_EBUSY if the queue
 * is full or the request alone exceeds the budget; KSS_ENOTSUP for atoms with an overlap Q. */
kss_status kss_server_submit(kss_ctx ctx, const kss_cell* cell, const kss_atoms* atoms, int nband,
                             uint64_t* ticket);

/* Drive the server from the calling thread for up to max_ms (at least one tick): each tick admits
 * what fits, runs one lockstep iteration over every unit in flight (new units start in the same
 * tick) and retires finished requests.  Returns early when idle.  in_flight / queued: requests
 * on the device / waiting (may be NULL).  Errors: KSS_EINVAL (no server), and device errors of
 * the lockstep engine (KSS_ENOMEM, KSS_ECUDA, KSS_ENUMERIC); a request whose own setup fails is
 * retired with that status instead (see kss_server_poll). */
kss_status kss_server_pump(kss_ctx ctx, double max_ms, int* in_flight, int* queued);

/* *done = 1 when the request finished; then evals / resid (host, nk*nband, k-point-major) and
 * the latency are filled and the ticket is released.  Returns the request's status once done
 * (KSS_OK, KSS_ENOCONV, or the setup error).  Errors: KSS_EINVAL (no server, unknown or already
 * collected ticket). */
kss_status kss_server_poll(kss_ctx ctx, uint64_t ticket, int* done, double* evals, double* resid,
                           double* latency_ms);

/* Counters and latency percentiles so far.  Errors: KSS_EINVAL (NULL, no server). */
kss_status kss_server_get_stats(kss_ctx ctx, kss_server_stats* out);

/* Stop the server and free everything it holds (pending and in-flight requests are dropped).
 * Errors: KSS_EINVAL (NULL, no server), KSS_ECUDA. */
kss_status kss_server_stop(kss_ctx ctx);

/* ------------------------------------------------------------------------------------------
 * Launch accounting and per-kernel timing (measurement support; no counterpart in the paper)
 * ------------------------------------------------------------------------------------------ */

/* Reset the context's counters; enable != 0 also brackets every later kernel launch of this
 * library with a pair of CUDA events on the context stream (small overhead per launch).
 * Errors: KSS_EINVAL (NULL). */
kss_status kss_profile_enable(kss_ctx ctx, int enable);

/* Number of kernel names seen so far (entries) and launches since the last reset.  Waits for
 * the context stream when timing is enabled.  Errors: KSS_EINVAL (NULL). */
kss_status kss_profile_count(kss_ctx ctx, int* nkernels, long long* launches);

/* Entry i < nkernels: kernel name (library-owned, static), launches and total event-timed
 * milliseconds since the last reset (0 when timing was off).  KSS_EINVAL past the end. */
kss_status kss_profile_entry(kss_ctx ctx, int i, const char** name, long long* launches,
                             double* total_ms);

/* ------------------------------------------------------------------------------------------
 * Autotuner of the FFT radix schedule (the batched pencil FFTs of §5.1; the schedule itself is
 * this library's choice, the paper fixes none)
 *
 * The y/z transforms of one x-plane (the middle pass of the local-potential path) have several
 * kernel schedules for a box length N: a split N = A * B into two register codelets
 * (A, B <= 16, e.g. 96 = 8 x 12, 12 x 8, 6 x 16, 16 x 6), spread over 256 or 384 threads per
 * CTA (also 128 in single precision), or a per-warp form.  With autotuning on, the first use of a (device, precision, box,
 * sphere window) configuration times every candidate on a scratch slab and keeps the fastest
 * for the rest of the process.  The candidates compute the same transform and differ only in
 * rounding order (results agree to a few ulps).  Tuning never runs inside a CUDA stream capture
 * or in kss_apply_H_noalloc; those use the table entry if one exists, else the built-in choice.
 * ------------------------------------------------------------------------------------------ */

/* mode 1 (default): tune at first use; mode 0: built-in choice for configurations not yet in
 * the table.  KSS_EINVAL for another mode. */
kss_status kss_autotune_set(kss_ctx ctx, int mode);

typedef struct {
  int device, precision;  /* precision: KSS_PREC_FP64 or KSS_PREC_MIXED */
  int N1, N, W3, W2;      /* box N1 x N x N and sphere window W2 x W3 of the configuration */
  int A, B, threads;      /* chosen split N = A * B; threads per CTA (0: per-warp form) */
  double ms;              /* time of one tuning launch of the chosen schedule */
  int ncand;              /* candidates timed */
} kss_tune_entry;

/* Number of table entries (process-wide, all contexts).  Errors: KSS_EINVAL (n == NULL). */
kss_status kss_autotune_count(int* n);
/* Entry i (insertion order); KSS_EINVAL past the end or for a NULL out. */
kss_status kss_autotune_get(int i, kss_tune_entry* out);
/* Insert or replace the entry for (device, precision, N1, N, W3 rounded up to a multiple of 8):
 * pins a schedule (e.g. one read back from an earlier run, for run-to-run identical rounding).
 * A, B, threads as in kss_tune_entry (ms, ncand, W2 ignored).  A pinned schedule without a
 * kernel instance, or whose shared memory does not fit a configuration's window, falls back to
 * the per-warp form at use.  KSS_EINVAL for inconsistent fields (A * B != N, threads not in
 * {0, 128, 256, 384}, W3 outside [1, N], unknown precision). */
kss_status kss_autotune_put(const kss_tune_entry* e);
/* Empty the tables of the FFT schedules and of the GEMM K-splits below (later configurations are
 * tuned again).  Cannot fail (returns KSS_OK). */
kss_status kss_autotune_clear(void);

/* The tensor-core GEMMs (the projector products, Eq. ham-nl of §5.2; the Gram and rotation
 * products of Rayleigh-Ritz, §5.1) split K across CTAs when a product has few output tiles, and the
 * split-BF16 products have three kernel forms: one CTA per 128 x 128 output tile (form 0), or
 * persistent CTAs (one per SM) that walk the output tiles with two TMEM accumulators, so that the
 * epilogue of one tile overlaps the MMAs of the next, on 128 x 128 (form 1) or 128 x 64 (form 2)
 * tiles.  With tuning on (kss_autotune_set), the first product of each (kind, shape) times the
 * candidate schedules (each form with no split, the closed-form plan, and the splits that fill the
 * SMs in one, two or three waves) on the device and keeps the fastest for the process; every
 * schedule computes the same product (the K ranges are added in a fixed order).  kind: 0
 * split-BF16 complex64 products, 1 FP64 digit products, 2 the same with a complex64 result, 3
 * 4-digit products of complex64 data.  Mr: real rows of the product (twice the complex rows), Nr:
 * columns, kblocks: K in k-blocks of the kernel. */
typedef struct {
  int device, kind, Mr, Nr, kblocks;
  int splits;  /* chosen K-split (CTAs along K) */
  double ms;   /* time of one tuning run of the chosen schedule (0 for a pinned entry) */
  int ncand;   /* candidates timed (0 for a pinned entry) */
  int form;    /* kernel form (kind 0: 0, 1 or 2 as above; other kinds: 0) */
} kss_gemm_tune_entry;

/* Number of GEMM K-split table entries (process-wide).  Errors: KSS_EINVAL (n == NULL). */
kss_status kss_autotune_gemm_count(int* n);
/* Entry i (insertion order); KSS_EINVAL past the end or for a NULL out. */
kss_status kss_autotune_gemm_get(int i, kss_gemm_tune_entry* out);
/* Insert or replace the entry for (device, kind, Mr, Nr, kblocks): pins a form and a split (the
 * split clamped at use to the kernel's minimum k-blocks per CTA).  ms and ncand are ignored.
 * Errors: KSS_EINVAL (NULL, kind outside 0..3, sizes < 1, splits outside [1, kblocks], form outside
 * 0..2 for kind 0 or not 0 for the other kinds). */
kss_status kss_autotune_gemm_put(const kss_gemm_tune_entry* e);

#ifdef __cplusplus
}
#endif
#endif /* KSS_H */
