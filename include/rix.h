/*
 * rix -- RI-LVL real-space exact-exchange build on one NVIDIA GB300 (sm_103a).
 *
 * C ABI of librix.so.  Plain pointers and sizes only; no C++ or framework
 * types cross this boundary.  Every entry point returns a rix_status and
 * never aborts; device-side work is enqueued on the caller's CUDA stream and
 * the compute entry points never synchronise the host.
 *
 * The operation (Kokott et al., arXiv:2403.10343, Sec. "Description of the
 * real-space formalism", Eq. 4 with the RI-LVL restriction of Eqs. 6-7):
 *
 *   K_il(n) = sum_{jk} sum_{PQ} C^P_ij V_PQ C^Q_kl D_jk
 *   E_x     = -1/4 sum_il D_li K_il            (-1/4 Tr(D K), one cell)
 *
 * i is a basis function of atom A in cell 0, l of atom E in cell n; P is an
 * auxiliary function on the atom of i or of j, Q on the atom of k or of l.
 *
 * ---------------------------------------------------------------------------
 * Block-sparse packed format (shared by C, V, D, K and the gradients)
 * ---------------------------------------------------------------------------
 * A pair (A, B, n1, n2, n3) joins atom A in cell 0 to atom B in cell
 * n = n1 a1 + n2 a2 + n3 a3.  The pair list holds every pair with
 * |x_B + n - x_A| < cutoff (every pair at n = 0 when cutoff <= 0, cluster only),
 * or the caller's list (rix_system.pairs), sorted lexicographically by
 * (A, B, n1, n2, n3); the cutoff list is exactly symmetric:
 * the distance is evaluated in the orientation with A < B (or A == B and
 * n > 0 lexicographically) as dx_c = (x_B,c + s_c) - x_A,c with
 * s_c = (n1 a1_c + n2 a2_c) + n3 a3_c and d^2 = (dx_0^2 + dx_1^2) + dx_2^2,
 * without fused multiply-add.
 *
 *   C(A,B,n): [P][i][j] row-major, P over aux(A) then aux(B) (aux(A) only for
 *             the on-site pair A == B, n == 0); i in basis(A), j in basis(B).
 *             Must satisfy C(B,A,-n)[P][j][i] == C(A,B,n)[P][i][j] bit for bit
 *             (the translational/pair symmetry the paper uses with Eqs. 11-12).
 *   V(A,B,n): [P][Q], P in aux(A), Q in aux(B at n); V(B,A,-n) = V(A,B,n)^T.
 *   D(A,B,n): [i][j]; D(B,A,-n) = D(A,B,n)^T (not checked).
 *   K(A,E,n): [i][l] on the K pattern: every (A, E, n) reachable from A by at
 *             most three pair hops (the reach of the four RI-LVL terms).
 *
 * Blocks are stored back to back in list order; rix_layout returns each
 * list's keys and element offsets.  A key packs (A, B, n) as
 * A << 44 | B << 24 | (n1+128) << 16 | (n2+128) << 8 | (n3+128).
 *
 * Input screening (paper Sec. "Initialization": compression of C and V
 * below 1e-10; Sec. "Evaluation of the EXX matrix": norm screening): a C,
 * V or D block whose largest |element| is below screen_tau contributes zero.
 *
 * Ownership: host arrays passed to rix_setup are copied.  Device buffers
 * passed to rix_set_CV are copied into library-owned storage.  D, K, E_x and
 * gradient buffers are caller-owned device memory that must stay valid until
 * the enqueued work has finished on the stream.  Everything else (pair lists,
 * plans, workspaces) is owned by the context and freed by rix_destroy.
 */
#ifndef RIX_H
#define RIX_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rix_ctx rix_ctx;

typedef enum {
  RIX_OK = 0,
  RIX_EINVAL = 1,        /* bad argument or inconsistent sizes */
  RIX_ENOMEM = 2,        /* device or host allocation failed, or plan exceeds the memory limit */
  RIX_ECUDA = 3,         /* a CUDA call failed; rix_last_error() has the message */
  RIX_ENOTSYM = 4,       /* C or V violates the pair symmetry */
  RIX_ETIMEOUT = 5,      /* a bounded device wait ran out */
  RIX_EUNSUPPORTED = 6,  /* valid request the library does not support */
  RIX_ESTATE = 7         /* call out of order (e.g. build before set_CV) */
} rix_status;

typedef enum {
  RIX_FP64 = 0,          /* every product and sum in IEEE double */
  RIX_MIXED_BF16 = 1     /* tensor-core products on error-free BF16 slices, FP64 sums */
} rix_precision;

/* Lists returned by rix_layout: the pair list with the C, V or D element
 * offsets, or the K list with the K offsets. */
enum { RIX_LIST_C = 0, RIX_LIST_V = 1, RIX_LIST_D = 2, RIX_LIST_K = 3 };

typedef struct {
  int32_t n_atoms;
  const double *xyz_bohr;          /* [n_atoms][3], host */
  const int32_t *species;          /* [n_atoms] species index, host */
  int32_t n_species;
  const int32_t *nbas_per_species; /* [n_species] basis functions (1..64) */
  const int32_t *naux_per_species; /* [n_species] aux functions (1..256) */
  const double *cell_bohr;         /* [3][3] rows = lattice vectors; NULL = cluster */
  double cutoff_bohr;              /* pair cutoff; <= 0 = all pairs (cluster only) */
  double screen_tau;               /* block screening threshold; <= 0 = none */
  int64_t n_pairs;                 /* optional caller-supplied pair list (0 / NULL: built from the cutoff) */
  const int32_t *pairs;            /* [n_pairs][5] = (A, B, n1, n2, n3), host, any order; it must be
                                      symmetric (with every (A,B,n) also (B,A,-n)), free of duplicates,
                                      with atoms in range, |n_c| <= 42 and n = 0 for a cluster (EINVAL
                                      otherwise, before any device work); the cutoff then only names the
                                      system, the list decides which blocks exist */
} rix_system;

typedef struct {
  int32_t precision;               /* rix_precision */
  int32_t n_slices;                /* mixed mode: BF16 slices per operand, 1..8 (0 = default, 5; the
                                      regrouped plans take one more) */
  int64_t max_workspace_bytes;     /* 0 = no limit beyond the device's free memory */
  int32_t verbose;                 /* 0 = silent */
  int32_t profile;                 /* 1 = record a CUDA event after every stage of rix_build_K
                                      (skipped while the stream is being captured into a graph);
                                      2 = also an event pair around every sliced-GEMM launch
                                      (rix_gemm_profile) */
  int32_t backward;                /* 1 = also plan rix_backward (extra product lists) */
  int32_t block_atoms;             /* > 0: row blocks of at most this many atoms (the paper's manual
                                      Fock-matrix block size); 0 = blocks only where memory requires */
  int32_t n_slices_regrouped;      /* mixed mode: slices of the regrouped plans (term 1 as T x C, the
                                      term-4 intermediate, T), 1..8; 0 = n_slices + 1 */
  int32_t reuse_forward;           /* rix_backward's recompute switch.  0 (default): recompute T, U2, Z
                                      and K from D.  1: when the plan has one row block and the
                                      preceding call on the context was rix_build_K with the same D
                                      pointer (the caller guarantees D and that K are unchanged since),
                                      reuse the intermediates and K that build left resident; otherwise
                                      recompute.  The adjoint overwrites them, so a second rix_backward
                                      recomputes. */
  double product_tau;              /* product screening (the paper's norm screening of block products,
                                      Sec. "Evaluation of the EXX matrix in real space"): a product of
                                      blocks whose max-norms multiply to less than product_tau is
                                      skipped -- C(A,B') D(B',G') in T, V(B,G') D(B,G') C(G',E') in Z
                                      (row tiles of V D on the tensor cores, against the largest C
                                      block of G').  An approximation whose error is the skipped
                                      products'; 0 = off (only input blocks below screen_tau are
                                      dropped).  The adjoint does not apply it. */
  int32_t deterministic;           /* mixed mode: 1 = bitwise reproducible builds.  The tensor-core
                                      contributions to K are added as 128-bit fixed-point integers
                                      (units of 2^-80, |K| < 2^47; integer addition does not depend on
                                      order) instead of FP64 atomics, and the term-4 intermediate runs
                                      on the output-stationary FP64 kernel.  (The FP64 path is always
                                      reproducible.) */
} rix_options;

typedef struct {
  int64_t n_atoms, n_pairs, n_pairs2, n_kblocks;
  int64_t c_elems, v_elems, d_elems, k_elems;
  double flops_fp64;               /* algorithmic FLOPs of one rix_build_K (unpadded products; terms 1
                                      and 4 counted once per pair / K block, as the build runs them) */
  double flops_stage[6];           /* T, U2, X12 (terms 1+2), Z (term 4), X34, symmetrise */
  double min_bytes;                /* 8 (nnz C + V + D) + 8 nnz K */
  double tensor_flops;             /* mixed mode: tensor-core FLOPs issued per build */
  int64_t workspace_bytes;         /* library-owned device memory */
  int32_t n_row_blocks;            /* row blocks of the memory plan (1 = all intermediates resident) */
  double flops_term2;              /* the term-2 part of flops_stage[2] (on the tensor cores when mixed) */
  double tensor_flops_stage[5];    /* mixed mode: tensor FLOPs issued per build for terms 3+4, term 2,
                                      term 1, term-4 intermediate Z, T */
  int32_t launches_build;          /* kernel launches of one rix_build_K (rix_energy adds 3) */
  double flops_term1_tc;           /* mixed mode: the term-1 FLOPs (FP64 grouping) moved to the tensor cores */
  double flops_z_tc;               /* mixed mode: the Z FLOPs (FP64 grouping) moved to the tensor cores */
  int64_t tz_bytes;                /* the T and Z buffers (part of workspace_bytes) */
  double flops_t_tc;               /* mixed mode: the T FLOPs moved to the tensor cores */
  int64_t nbasis;                  /* basis functions per cell (the side of rix_fold_gamma's matrix) */
} rix_stats_t;

/* Set up a system: copies the host arrays, builds the pair list on the device
 * (a1: cutoff over image-resolved pairs), derives the 2- and 3-hop lists and
 * the product plan, and allocates workspaces.  Synchronous.  Errors: EINVAL
 * (sizes, species tables, periodic without cutoff, images beyond +-127),
 * ENOMEM, ECUDA.  On error *out is NULL. */
rix_status rix_setup(const rix_system *sys, const rix_options *opt, rix_ctx **out);

/* Host views of a list: number of blocks, keys [n] and element offsets [n+1]
 * (block b occupies [offsets[b], offsets[b+1]) of the packed array).  which
 * is one of RIX_LIST_C/V/D (same keys, per-array offsets) or RIX_LIST_K.
 * The arrays belong to the context and live until rix_destroy. */
rix_status rix_layout(const rix_ctx *ctx, int32_t which, int64_t *n_blocks,
                      const int64_t **keys, const int64_t **offsets);

/* Element counts of the packed C, V, D and K arrays. */
rix_status rix_layout_sizes(const rix_ctx *ctx, int64_t *c_elems, int64_t *v_elems,
                            int64_t *d_elems, int64_t *k_elems);

/* Load C and V (packed format, FP64).  Each pointer may be device memory or
 * host memory (pinned or pageable; the copy direction follows from the
 * address), so a caller whose C does not fit twice on the device can load it
 * straight from the host.  Copies them into library storage, checks the pair
 * symmetry of C and V (ENOTSYM), computes the screening flags and, in mixed
 * mode, the BF16 slices.  Enqueued on `stream` (cudaStream_t, NULL = legacy
 * default stream); synchronises the stream once to read the symmetry
 * verdict. */
rix_status rix_set_CV(rix_ctx *ctx, const double *C_dev, const double *V_dev, void *stream);

/* Autotuner (no counterpart in the paper's code path beyond its auto-tuned
 * Fock-matrix block size): picks the shared-memory tile budget of the three
 * FP64 contraction kernels (terms 1+2, the term-4 intermediate Z, terms 3+4)
 * by timing four candidates on a slice of this system's own work items with
 * the density matrix D_dev (device, packed).  Needs rix_set_CV first.
 * cache_path (may be NULL): a text file of "key x12 z x34" lines; a line
 * whose key (device name and list sizes) matches is applied without timing,
 * and a new choice is appended.  chosen (may be NULL) receives the three
 * budgets in doubles.  Synchronises `stream`; not allowed during graph
 * capture (RIX_ESTATE).  Results of later builds change only by rounding. */
rix_status rix_autotune(rix_ctx *ctx, const double *D_dev, const char *cache_path, int32_t *chosen,
                        void *stream);

/* K = exchange matrix of D (device, packed, FP64) into K_dev (device, packed
 * on the K list, FP64, fully overwritten): Eq. 4 with the RI-LVL restriction
 * of Eqs. 6-7, evaluated in the four-term grouping of Eq. 11 and Eqs. 12a-d.
 * D must be pair-symmetric, D(B,A,-n) = D(A,B,n)^T, as a density matrix is:
 * K is formed as X + X^T with term 3 taken as the transpose of term 2 and
 * terms 1 and 4 evaluated for one orientation of each block, all of which
 * rest on that symmetry (C and V are checked by rix_set_CV; D is not).
 * Asynchronous on `stream`; no host synchronisation, no allocation; may be
 * captured in a CUDA graph once one call has completed.  ESTATE before
 * rix_set_CV. */
rix_status rix_build_K(rix_ctx *ctx, const double *D_dev, double *K_dev, void *stream);

/* Incremental build for the SCF loop (the paper's exchange matrix is rebuilt
 * from the unmixed density every iteration, Sec. "Evaluation of the EXX
 * matrix in real space"): K_dev += K(dD_dev), with dD = D_new - D_old in the
 * packed D layout.  K is linear in D, so K(D_old) + K(dD) = K(D_new); blocks
 * of dD below screen_tau are skipped like blocks of D, so once the density
 * settles most of dD is screened out and the build does less work.  The same
 * stages, precision and synchronisation behaviour as rix_build_K
 * (asynchronous, no allocation, graph-capturable); K_dev is read and
 * updated. */
rix_status rix_build_K_delta(rix_ctx *ctx, const double *dD_dev, double *K_dev, void *stream);

/* *Ex_dev = -1/4 sum over the D pattern of <D(E,A,-n), K(A,E,n)>_F, a
 * deterministic FP64 tree reduction.  Ex_dev is one device double. */
rix_status rix_energy(rix_ctx *ctx, const double *D_dev, const double *K_dev,
                      double *Ex_dev, void *stream);

/* The same energy as rix_energy, for callers that must not allocate device
 * memory when they ask for it (a framework whose caching allocator already
 * holds the GPU's free memory, or an SCF loop that forbids allocation and the
 * synchronisation it can cause).  No counterpart in the paper: it only moves
 * the reduction's scratch (one partial sum per 256 pairs) into a fixed
 * 512 KB device array owned by the library (kept on every GPU that loads it
 * until exit).  Contexts with more than 16,777,216 pairs are rejected
 * (RIX_EINVAL).  Every call on a device shares that array: calls whose work
 * overlaps on the GPU race.  rix_setup looks up the array's address with the
 * context's device current, so this call makes no CUDA runtime call besides
 * its kernel launches.  Asynchronous. */
rix_status rix_energy_noalloc(rix_ctx *ctx, const double *D_dev, const double *K_dev,
                              double *Ex_dev, void *stream);

/* Adjoint of E_x scaled by gEx (host scalar): dD_dev [d_elems] = gEx * dE/dD
 * = -gEx K(D)/2 per stored D entry, dC_dev [c_elems] = gEx * dE/dC per stored
 * C entry, dV_dev [v_elems] = gEx * dE/dV per stored V entry (partials with
 * every stored entry an independent variable; symmetric partners each carry
 * their own).  Any output pointer may be NULL to skip it.  Intermediates are
 * recomputed, not stored.  Asynchronous. */
rix_status rix_backward(rix_ctx *ctx, const double *D_dev, double gEx,
                        double *dD_dev, double *dC_dev, double *dV_dev, void *stream);

/* Force and stress chain of E_x (the paper's Secs. "EXX force and stress
 * contributions" and "Computation of Forces and Stress"), one Cartesian
 * component c (0, 1, 2) per call, the paper's split of this work into three
 * parts to bound memory.  C(A,B,n) and V(A,B,n) depend on the geometry
 * through the pair vector r_p = x_B + n . a - x_A.  Inputs (device, packed):
 * dEdC [c_elems], dEdV [v_elems] from rix_backward (either may be NULL to
 * leave that part out), and the caller's derivatives of the stored C and V
 * entries with respect to component c of their pair's r_p, dCdr_c
 * [c_elems], dVdr_c [v_elems].  With g_p = sum_e dE/dC_pe dC_pe/d(r_p)_c
 * (+ the V part):
 *   F_dev[X]   = -dE/dx_X,c = sum over the pairs p = (X, B, n) of (g_p - g_(B,X,-n))
 *                (n_atoms doubles, overwritten; may be NULL)
 *   stress_dev = row c of (1/Omega) dE/d eps, eps the homogeneous strain that maps
 *                every r_p to (1 + eps) r_p: stress_dev[b] = (1/Omega) sum_p g_p (r_p)_b
 *                (3 doubles, overwritten; periodic only, may be NULL).
 * D is held fixed (its own geometry dependence belongs to the SCF).  Fixed
 * summation order (deterministic); asynchronous; no allocation. */
rix_status rix_force_stress(rix_ctx *ctx, int32_t c, const double *dEdC_dev, const double *dEdV_dev,
                            const double *dCdr_c_dev, const double *dVdr_c_dev, double *F_dev, double *stress_dev,
                            void *stream);

/* RI-LVL coefficient fit (the paper's Eq. 8 with the pair-restricted Coulomb
 * metric of Eq. 10; part of its "Initialization" stage, once per geometry):
 *   C(I,J,n)^mu_ij = sum_{nu in P(IJ)} (ij|nu) [(V^{IJ} + lambda 1)^{-1}]_{nu mu}
 * with P(IJ) = aux(I) then aux(J) (aux(I) alone on-site), V^{IJ} assembled
 * from the on-site blocks V(I,I,0), V(J,J,0) and the pair block V(I,J,n).
 * V_dev: packed V (RIX_LIST_V layout), eri_dev: the three-centre integrals
 * (ij|nu) in the packed C layout, C_dev: output, packed C (all device).  Each
 * representative pair is factored by Cholesky and solved on the device; its
 * partner receives the transposed numbers, so C is exactly pair-symmetric
 * (rix_set_CV accepts it).  lambda >= 0 shifts the metric's diagonal (a
 * Tikhonov fit) for metrics that are numerically singular; EINVAL if a shifted
 * metric is still not positive definite.  Allocates its workspace (up to
 * 1 GB) on `stream` and synchronises it. */
rix_status rix_fit_C(rix_ctx *ctx, const double *V_dev, const double *eri_dev, double lambda, double *C_dev,
                     void *stream);

/* Gamma-point fold of an image-resolved K: Kdense[I][L] = sum_n K(A,E,n)[i][l]
 * (I, L global basis indices), row-major nbasis x nbasis.  Asynchronous. */
rix_status rix_fold_gamma(rix_ctx *ctx, const double *K_dev, double *Kdense_dev, void *stream);

/* Bloch sums of an image-resolved K (the paper's Eq. 3, Fock operator in k
 * space): for each of the n_k points kappa (host, [n_k][3], fractional
 * coordinates in the reciprocal basis b_c with b_c . a_d = 2 pi delta_cd),
 *   Kk[q][I][L] = sum_n exp(2 pi i kappa_q . n) K(A,E,n)[i][l]
 * (I, L global basis indices).  K_dev: packed on the K list (device); Kk_dev:
 * device, n_k consecutive row-major nbasis x nbasis complex matrices stored
 * as interleaved (re, im) doubles, fully overwritten.  kappa = 0 gives the
 * Gamma fold of rix_fold_gamma with zero imaginary parts.  A cluster accepts
 * only kappa = 0 (EINVAL otherwise).  Asynchronous; one kernel per k point. */
rix_status rix_bloch(rix_ctx *ctx, const double *K_dev, int32_t n_k, const double *kfrac, double *Kk_dev,
                     void *stream);

/* Collinear spin (the spin index sigma of the paper's Eqs. 3-5; the spin
 * channels double the work): D_dev holds n_spin (1 or 2) packed densities back
 * to back (d_elems each, the per-spin density matrices D^up, D^dn without the
 * closed-shell factor 2), K_dev receives n_spin packed K arrays (k_elems
 * each): K^sigma = K(D^sigma), one build per channel.  Asynchronous. */
rix_status rix_build_K_spin(rix_ctx *ctx, int32_t n_spin, const double *D_dev, double *K_dev, void *stream);

/* Exchange energy of spin-resolved D and K (layout as rix_build_K_spin):
 * E_x = -1/2 sum_sigma Tr(D^sigma K^sigma) for n_spin = 2 (equal to -1/4
 * Tr(D K) of the closed shell when D^up = D^dn = D/2), -1/4 Tr(D K) for
 * n_spin = 1.  Ex_dev: one device double.  Asynchronous. */
rix_status rix_energy_spin(rix_ctx *ctx, int32_t n_spin, const double *D_dev, const double *K_dev, double *Ex_dev,
                           void *stream);

/* C = A B for FP64 device matrices (row-major, leading dimensions in elements;
 * C overwritten) computed on the BF16 tensor cores by error-free slicing: each
 * row of A and column of B is scaled by its own power of two and written with
 * n_slices (1..8) balanced base-2^7 digits (the last rounded to nearest); the
 * slice products with s + t <= n_slices + 1 are accumulated exactly and
 * combined in 64-bit fixed point.  Error about 2^(-7 n_slices - 1) of (row
 * scale x column scale x K) (measured 2^-45.2 at 6 slices).  The splitting
 * is Ozaki, Ogita, Oishi, Rump (2012); the paper itself uses FP64 BLAS
 * (Sec. "Improvements of other relevant code parts").  Allocates its slice
 * buffers on `stream` and synchronises it.  ETIMEOUT if a device wait ran out. */
rix_status rix_gemm_sliced(const double *A, int64_t lda, const double *B, int64_t ldb, double *C,
                           int64_t ldc, int32_t M, int32_t N, int32_t K, int32_t n_slices, void *stream);

/* Test hook for the bounded waits (no counterpart in the paper): runs the
 * sliced-GEMM kernel on a small zero problem (M = 130, N = 90, K = 70, three
 * slices) whose MMA issuer waits on a shared-memory barrier that nothing
 * completes; every wait of the launch gives up after wait_ns (1 .. 2e9), the
 * kernel waits for its own bulk copies, frees its tensor memory and records the
 * timeout.  ctx == NULL: synchronises `stream` and returns RIX_ETIMEOUT when
 * that path worked.  ctx != NULL: the kernel records the timeout in the
 * context's status word, the call returns RIX_OK without synchronising, and
 * rix_check (or the context's next entry point) reports RIX_ETIMEOUT.  The
 * stream and the CUDA context stay usable either way.  RIX_EINVAL for a
 * wait_ns out of range.  Allocates its operands on `stream`. */
rix_status rix_test_stalled_gemm(rix_ctx *ctx, int64_t wait_ns, void *stream);

/* Synchronises `stream` and reports the device-side status of the context:
 * RIX_ETIMEOUT if a bounded wait of one of its kernels gave up since the last
 * report (the results of that call are invalid; the flag is then cleared),
 * RIX_ECUDA if the stream holds a CUDA error.  rix_build_K, rix_energy,
 * rix_energy_noalloc, rix_backward and rix_set_CV make the same report at
 * entry for work that has already completed.  ESTATE inside a graph capture. */
rix_status rix_check(rix_ctx *ctx, void *stream);

rix_status rix_stats(const rix_ctx *ctx, rix_stats_t *out);

/* Algorithmic FLOPs (2 per multiply-add, the FP64 grouping of Eqs. 12a-d) that
 * one rix_build_K with the density matrix D_dev (device, packed) performs
 * after block screening (Sec. "Screening": products whose C, V or D block has
 * no element of magnitude >= tau are skipped).  Terms 1 and 4 are symmetric
 * under the transposition of their block (Eq. 11), so the build evaluates them
 * for one orientation of each pair / K block and these counts do the same.  The counts of rix_stats_t
 * include every product; these depend on D.  flops (host, 10 doubles):
 * [0] T, [1] U2, [2] terms 1+2, [3] Z, [4] terms 3+4, [5] symmetrise, [6] the
 * term-2 part of [2], [7] the part of [2] for the column atoms whose term 1
 * runs on the tensor cores, [8] the part of [3] for the middle atoms whose Z
 * products run on the tensor cores, [9] the part of [0] for the row atoms
 * whose T runs on the tensor cores ([7]-[9] are 0 in FP64 mode; the tensor
 * cores themselves do not skip screened products).  Needs rix_set_CV.
 * Synchronises `stream`; ESTATE inside a graph capture. */
rix_status rix_count_flops(rix_ctx *ctx, const double *D_dev, double *flops, void *stream);

/* Device time of each stage of rix_build_K (ms), summed over the builds since
 * the previous call, and the number of builds: ms[0..7] = screening flags,
 * T, U2, terms 1+2 (FP64 kernel), terms 1 and 2 on the tensor cores (mixed
 * only), Z, terms 3+4, symmetrise.  With several row blocks the T and U2
 * entries cover the first block and the terms 1+2 entry the rest of that
 * loop (including the tensor-core term 1 of those blocks); the Z entry
 * likewise covers the first block.  Needs rix_options.profile = 1
 * (the events are recorded on the build's stream); synchronises on the last
 * recorded event.  EUNSUPPORTED without profiling. */
rix_status rix_stage_times(rix_ctx *ctx, double *ms, int32_t n, int32_t *n_builds);
/* Per-kernel measurement of the tensor-core GEMM (needs rix_options.profile = 2
 * and mixed precision): device time of every k_gemm_sliced launch enqueued
 * since the previous call, from the event pairs around each launch (none are
 * recorded while a stream is being captured), summed into *ms; *launches the
 * number of launches; *chunks the MMAs they issued (one 128 x 80 x 16 product
 * of one slice pair each), so that the BF16 FLOPs issued are
 * *chunks x 2 x 128 x 80 x 16.  Synchronises on the last event; resets the
 * counts.  EUNSUPPORTED otherwise. */
rix_status rix_gemm_profile(rix_ctx *ctx, double *ms, int64_t *launches, int64_t *chunks);

const char *rix_strerror(rix_status s);
const char *rix_last_error(const rix_ctx *ctx);
void rix_destroy(rix_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* RIX_H */
