/*
 * bse.h - C ABI of the GB300 (sm_103a) plane-wave Bethe-Salpeter hot path.
 *
 * The path (Yan, Jacobsen & Thygesen, "Optical properties of bulk
 * semiconductors and graphene/boron nitride", Sec. II C, Sec. III A and
 * Appendix A) computes, for one or more periodic systems:
 *
 *   A0  plane-wave spheres, q folding, e-h pair and block tables (host)
 *   A1  u_nk(r) = sum_G c_nk(G) exp(iG.r) on the real-space grid       (Eq. pair_density)
 *   A2  rho_nm^{kk'}(G) on the q sphere: plane-wave correlation (default) or
 *       pruned FFT of conj(u_nk) u_mk' (the paper's route)           (Eq. pair_density)
 *   A3  K^x = rho_x^H diag(vbar) rho_x / (Omega Nk)                   (Eq. V_eh, G = 0 dropped)
 *   A4  K^d = rho_vv'^H W(q) rho_cc' / (Omega Nk) per (k,k') block      (Eq. W_SS)
 *   A5  H = diag(e_c + Delta - e_v) + 2 K^x - K^d  (TDA, Eq. kernel)
 *   A6  k.p dipole P_S (Eq. density_matrix)
 *   A7  Haydock/Lanczos recursion on H from P (FP64 recurrence)
 *   A8  eps_2(w) = -C |P|^2 Im g(w + i eta), C = 8 pi/(Omega Nk)     (Eq. epsilon_chi_bar)
 *   A9  adjoint of a spectral loss w.r.t. Delta, W and the pair densities
 *
 * Conventions (all entry points):
 *  - Hartree atomic units.  Complex single = interleaved float2 (re, im),
 *    complex double = interleaved double2.
 *  - Every pointer argument except the plan, the info structs and the
 *    explicitly host arrays is a DEVICE pointer owned by the caller; the
 *    library never frees caller memory and never allocates after
 *    bse_plan_create.  Scratch comes from a caller-allocated workspace whose
 *    size bse_workspace_size reports.
 *  - Calls enqueue work on the given stream and return without a host
 *    synchronisation; errors detected on the host are returned at once,
 *    errors detected on the device land in the plan's device status word and
 *    are returned by bse_status_read (which synchronises the stream).
 *  - Every function returns a bse_status; bse_last_error() gives a
 *    thread-local message for the last non-OK status.
 *  - Non-finite inputs: each compute call first streams its caller-supplied
 *    floating-point inputs (coef, energies, the W rows of its q range, H, A, B,
 *    X, P, omega, dL_deps2, W_ibz) through a device scan; a NaN or an infinity
 *    sets BSE_ERR_NONFINITE in the plan's device status word (returned by
 *    bse_status_read), and the outputs of that call are then undefined.  The
 *    pair densities and other library-produced intermediates are not scanned.
 *  - Systems inside one plan are addressed by index s in [0, nsys).
 */
#ifndef BSE_H
#define BSE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  BSE_OK = 0,
  BSE_ERR_ARG = 1,          /* invalid argument, shape or size */
  BSE_ERR_CUDA = 2,         /* CUDA runtime error (message in bse_last_error) */
  BSE_ERR_NONFINITE = 3,    /* NaN/Inf found in an input scan */
  BSE_ERR_TIMEOUT = 4,      /* a bounded device-side wait gave up */
  BSE_ERR_UNSUPPORTED = 5,  /* configuration outside the compiled kernels */
  BSE_ERR_WORKSPACE = 6,    /* workspace smaller than bse_workspace_size */
  BSE_ERR_INDEFINITE = 7    /* coupled spectrum: F H2 not positive definite (unstable system) or P = 0 */
} bse_status;

typedef enum { BSE_LATTICE_FCC = 0, BSE_LATTICE_HEX = 1 } bse_lattice;
typedef enum { BSE_COULOMB_3D = 0, BSE_COULOMB_SLAB = 1 } bse_coulomb;
typedef enum { BSE_PREC_FP32 = 0, BSE_PREC_BF16X3 = 1 } bse_precision;

/* Workspace kinds for bse_workspace_size. */
typedef enum {
  BSE_WS_PAIR = 0,      /* bse_pair_densities: real-space wavefunctions u_nk(r) */
  BSE_WS_KERNEL = 1,    /* bse_build_kernel: W.rho products of one q chunk */
  BSE_WS_SPECTRUM = 2,  /* bse_spectrum: Krylov basis, vectors, partial sums */
  BSE_WS_BACKWARD = 3,  /* bse_spectrum_backward: basis, dL/dH, chain products */
  BSE_WS_SCREEN = 4,    /* bse_screening: dielectric matrices of one q chunk (arg = chunk) */
  BSE_WS_COUPLING = 5,  /* bse_build_coupling: W.rho_cv' of one q chunk (arg = chunk; 0 = INIT only) */
  BSE_WS_COUPLED = 6,   /* bse_spectrum_coupled: basis, vectors, partial sums (arg = nsteps) */
  BSE_WS_RITZ = 7,      /* bse_ritz: per-Ritz-value scratch (arg = nsteps <= 4096; plan/system unused) */
  BSE_WS_CHI0 = 8,      /* bse_chi0_optical: pair vectors of the optical response */
  BSE_WS_ALDA = 9,      /* bse_xc_kernel_alda: f_xc(r) and the transform passes */
  BSE_WS_EPSM = 10,     /* bse_epsilon_macro: augmented Dyson systems (arg = nw) */
  BSE_WS_STATES = 11    /* bse_exciton_states: Krylov basis, tridiagonal eigenvectors (arg = n) */
} bse_ws_kind;

/* Stage flags for bse_pair_densities and bse_build_kernel. */
#define BSE_PD_REALSPACE 1u   /* A1: fill u_nk(r) in the workspace            */
#define BSE_PD_EXCHANGE  2u   /* A2 exchange set rho_x and the A6 dipole P     */
#define BSE_PD_DIRECT    4u   /* A2 direct set rho_vv', rho_cc' of a q range   */
#define BSE_PD_CHI0      8u   /* rho_vc^{k,k+q} for all k, q of a range (screening input) */
#define BSE_PD_COUPLING 16u   /* rho_vc', rho_cv' of the upper blocks of a q range (coupling) */
#define BSE_PD_TENSOR   32u   /* with DIRECT: the direct set on the tensor cores (BF16x3)      */
#define BSE_BK_INIT      1u   /* A3 + A5 diagonal: H = diag + 2 K^x (upper)    */
#define BSE_BK_DIRECT    2u   /* A4 + A5: H -= K^d for a q range, mirror       */
#define BSE_BK_MIRROR    4u   /* A5 without A4: lower blocks and (B+B^H)/2      */
#define BSE_BK_SYMFILL   8u   /* k-point symmetry: copy every other block from its representative */
#define BSE_BC_INIT      1u   /* coupling: B = 2 Bx (upper block triangle)       */
#define BSE_BC_DIRECT    2u   /* coupling: B -= Bd for a q range, mirror B^T     */
#define BSE_BC_MIRROR    4u   /* coupling without Bd: lower blocks, (B+B^T)/2    */

/*
 * One periodic system.  Lattices: fcc with conventional constant a
 * (a_i = a/2 {(0,1,1),(1,0,1),(1,1,0)}), or a hexagonal sheet a_1 = a(1,0,0),
 * a_2 = a(-1/2, sqrt3/2, 0), a_3 = (0,0,c).  k mesh Gamma-centred,
 * k = sum_j (i_j/nk_j) b_j, ik = (i1*nk2 + i2)*nk3 + i3; fcc needs
 * nk1 = nk2 = nk3, hex needs nk1 = nk2 and nk3 = 1.  The q mesh is the k mesh
 * (Sec. III A).  Spheres: |k+G|^2/2 <= ecut (wavefunctions) and |q+G|^2/2 <= ecut
 * (pair densities, W), ordered by exact key then g1, g2, g3.
 */
typedef struct {
  int lattice;          /* bse_lattice */
  double a;             /* bohr */
  double c;             /* bohr, hex out-of-plane period (ignored for fcc) */
  int nk[3];
  int nv, nc;           /* valence / conduction bands kept (TDA pair basis) */
  double ecut;          /* Ha */
  int fft[3];           /* real-space grid; each a divisor of 192 (2^a 3^b, b <= 1), <= 64 */
  int coulomb;          /* bse_coulomb: 3D 4pi/|G|^2 or slab-truncated 2D */
  double qhat[3];       /* optical-limit direction (Cartesian, normalised by the library) */
  double gap_floor;     /* Ha, floor of e_c - e_v in the dipole denominator */
  int kpoint_symmetry;  /* 1: the states carry the lattice's point group (psi_{Rk}(r) = psi_k(R^-1 r),
                           energies shared by each orbit) and W carries it too; the plan then keeps only
                           the representative upper blocks (see BSE_BK_SYMFILL).  0: every upper block. */
} bse_system;

/* Sizes and strides of system s (filled by bse_plan_info). */
typedef struct {
  int nkpt, nb, dim;          /* dim = nkpt*nv*nc, pair index S = (ik*nv + iv)*nc + ic */
  int npw_max;                /* coefficient row stride (max sphere size over k) */
  int ng_max;                 /* W row stride and pair-density vector stride */
  int ng0;                    /* size of the q = 0 sphere (exchange set) */
  int nq;                     /* = nkpt */
  long long nblocks;          /* upper (k <= k') blocks the plan builds (the representatives with k-point symmetry) */
  double omega_cell;          /* bohr^3 */
  double norm;                /* 1/(Omega Nk) */
  double prefactor;           /* C = 8 pi/(Omega Nk) */
  int kpoint_symmetry;        /* the system's bse_system.kpoint_symmetry */
  long long nfill;            /* upper blocks copied by BSE_BK_SYMFILL (0 without k-point symmetry) */
  int tensor_pair;            /* 1: BSE_PD_TENSOR is available for this system */
  int tc_region[3];           /* k' points per region of the tensor route (mesh axes 1-3) */
  int tc_kpad;                /* K layout length of the tensor route (padded to 32) */
} bse_info;

typedef struct bse_plan bse_plan;

/* Thread-local message of the last failing call (never NULL). */
const char* bse_last_error(void);

/*
 * A0.  Build host tables for nsys systems (Sec. II C plane-wave sets, Sec.
 * III A q mesh and G0 folding), upload them, and allocate the plan's small
 * device tables on the current device.  Errors: BSE_ERR_ARG for an invalid
 * system (lattice/mesh mismatch, grid not 2^a 3^b or too small for alias-free
 * pair densities: N_i > 2 Fwf_i + Fpair_i), BSE_ERR_CUDA on allocation
 * failure.  The plan is bound to the device current at creation.
 */
bse_status bse_plan_create(const bse_system* sys, int nsys, bse_plan** out);

/*
 * A0 on the host only: the same tables without any device allocation (no GPU
 * needed).  Such a plan serves bse_plan_info, the table exports and
 * bse_workspace_size / bse_rho_dir_count; compute calls return BSE_ERR_ARG.
 */
bse_status bse_plan_create_host(const bse_system* sys, int nsys, bse_plan** out);
bse_status bse_plan_destroy(bse_plan* plan);
bse_status bse_plan_info(const bse_plan* plan, int s, bse_info* info);

/*
 * Test exports of the bit-exact host tables (host buffers).
 * bse_gvectors: sphere of k (is_q = 0) or q (is_q = 1) of mesh index kq as
 * int32 [n][3] reduced G; pass out = NULL to query n.
 * bse_pair_blocks: the upper blocks of q-index iq in processing order as
 * int32 [n][2] (ik, ik'), plus G0 of each block as int32 [n][3]; out/g0 may be
 * NULL to query n.
 */
bse_status bse_gvectors(const bse_plan* plan, int s, int kq, int is_q, int32_t* out, int* n);
bse_status bse_pair_blocks(const bse_plan* plan, int s, int iq, int32_t* out, int32_t* g0, int* n);

/*
 * Workspace bytes for one call kind on system s.  For BSE_WS_KERNEL, arg is
 * the largest q chunk (q_end - q_begin) that will be passed; for
 * BSE_WS_SPECTRUM and BSE_WS_BACKWARD, arg is nsteps.  Ignored otherwise.
 */
bse_status bse_workspace_size(const bse_plan* plan, int s, int kind, long long arg, size_t* bytes);

/* Number of complex vectors of rho_dir for q in [q_begin, q_end) (each ng_max long). */
bse_status bse_rho_dir_count(const bse_plan* plan, int s, int q_begin, int q_end, long long* nvec);

/*
 * A1 + A2 (+ A6).  Pair densities (Eq. pair_density):
 *   rho_nm^{kk'}(G) = (1/N_r) sum_r conj(u_nk(r)) u_mk'(r) exp(-iG.r)
 *                   = sum_{G2 in S(k')} conj(c_nk(G2 - G)) c_mk'(G2).
 * Two routes give the same densities to FP32 rounding (bse_pair_variants): the
 * plane-wave correlation kernel (second form; the default wherever its band counts
 * are compiled) and the pruned batched 3D FFT of the products on the real-space
 * grid (first form; the default otherwise).
 * coef     complex64 [nkpt][nb][npw_max], c_nk(G) in sphere order (zero padded).
 * energies float64  [nkpt][nb], bands ascending (valence first), Ha.
 * rho_x    complex64 [dim][ng_max]: rho_vc^{kk}(G) on the q = 0 sphere (S = (k,v,c)).
 * P        complex128 [dim]: P_S = conj(qhat.sum_G conj(c_vk)(k+G)c_ck)/max(e_c-e_v, gap_floor).
 * rho_dir  complex64 [nvec][ng_max] for q in [q_begin, q_end): per q, first the
 *          nblk_q*nv*nv vectors rho~_vv'^{kk'} (block-major, then v, v'), then the
 *          nblk_q*nc*nc vectors rho~_cc'^{kk'} (nblk_q: the plan's blocks of q - with k-point
 *          symmetry only the representatives); entry p is taken at G = g_p(q) - G0,
 *          g_p the p-th vector of the q sphere, so q_unf + G = q + g_p.
 * flags    BSE_PD_* stages; REALSPACE must run (once) before the others, with
 *          the same workspace.  Unused outputs may be NULL.  With BSE_PD_COUPLING (not with
 *          DIRECT or CHI0) rho_dir receives the coupling densities of bse_build_coupling,
 *          bse_rho_cpl_count(q_begin, q_end) vectors.
 *          With BSE_PD_DIRECT | BSE_PD_TENSOR the direct set is computed on the tensor cores: for
 *          each k, the blocks whose k' lie in one region of the k' mesh (bse_info.tc_region points)
 *          form one GEMM per band n, D[G][(k', m)] = sum_{G2} conj(c_nk(G2 - G)) c_mk'(G2), rows G the
 *          union of the blocks' q spheres, K the union of the region's spheres S(k'), operands split
 *          hi + lo in BF16 with hi.hi + hi.lo + lo.hi accumulated in FP32 (relative error ~1e-5 of
 *          the largest density instead of FP32 rounding); the G = 0 overlaps of the diagonal blocks
 *          are summed in FP64.  Same layout and vectors as without the flag.  The precision of the
 *          mixed build (bse_build_kernel with BSE_PREC_BF16X3); no counterpart in the paper, which
 *          computes the densities by FFT.
 * Errors: BSE_ERR_ARG (range, NULL for a requested output), BSE_ERR_WORKSPACE, BSE_ERR_UNSUPPORTED
 *         (BSE_PD_TENSOR where bse_info.tensor_pair = 0), BSE_ERR_TIMEOUT (a tensor-route wait that
 *         did not end within 2 s, through the status word).
 */
bse_status bse_pair_densities(bse_plan* plan, int s, unsigned flags,
                              const void* coef, const double* energies,
                              void* rho_x, void* P,
                              void* rho_dir, int q_begin, int q_end,
                              void* ws, size_t ws_bytes, void* stream);

/*
 * A3 - A5.  Hamiltonian in the TDA (Eq. kernel, Eqs. V_eh and W_SS):
 *   H = diag(e_ck + delta - e_vk) + 2 K^x - K^d.
 * BSE_BK_INIT writes diag + 2K^x on the upper block triangle (k <= k') (on 128 x 128 tiles: also the
 * lower entries of the diagonal tiles, which DIRECT, MIRROR or SYMFILL then overwrite).  With
 * BSE_PREC_BF16X3 and a workspace (ws, at least bse_workspace_size(BSE_WS_KERNEL) for any chunk)
 * 2K^x = Y^H Y, Y = rho_x diag(sqrt(2 vbar/(Omega Nk))), is a BF16x3 tcgen05 Gram product; with
 * ws = NULL it is FP32 on CUDA cores.
 * BSE_BK_DIRECT subtracts K^d for the upper blocks of q in [q_begin, q_end)
 * (rho_dir laid out as in bse_pair_densities for the same range) and writes the
 * mirrored lower block H_k'k = H_kk'^H; diagonal blocks become (B + B^H)/2.
 * After INIT and DIRECT over all q, H is the full Hermitian matrix.
 * BSE_BK_MIRROR (not with DIRECT) completes an INIT-only build the same way: lower blocks
 * H_k'k = H_kk'^H, diagonal blocks (B + B^H)/2.  INIT | MIRROR is the Tamm-Dancoff form of the
 * random-phase response with local fields (exchange kernel only, no W).
 * k-point symmetry (bse_system.kpoint_symmetry = 1; Sec. III A: the pair densities of (k, k') equal
 * those of (Tk, Tk') on rotated G, so with symmetric states and W every block H_{Tk,Tk'} equals H_{k,k'}):
 * the plan's blocks (bse_pair_blocks, bse_rho_dir_count, bse_plan_info nblocks) are only the
 * representatives - the upper blocks in row-major order, each unassigned one a representative of
 * the blocks (R k, R k') that the operations R (identity first, then ascending row-major entries)
 * map it to, as the upper block itself when R k <= R k' and as its Hermitian mirror otherwise.
 * DIRECT then builds only those; BSE_BK_SYMFILL (after every DIRECT chunk) copies each other upper
 * block from its representative (or the representative's conjugate transpose) and writes its mirror.
 * The coupling build and the adjoint need every block and return BSE_ERR_UNSUPPORTED for such plans.
 * W        complex64 [nq][ng_max][ng_max], W_q[p][p'] Hermitian, including 4 pi.
 * H        complex64 [dim][dim] row-major.
 * prec     BSE_PREC_FP32 (CUDA-core FP32) or BSE_PREC_BF16X3 (tcgen05 BF16
 *          hi/lo split products, FP32 accumulation) for the contractions.
 * Errors: BSE_ERR_ARG, BSE_ERR_UNSUPPORTED (precision not built), BSE_ERR_WORKSPACE.
 */
bse_status bse_build_kernel(bse_plan* plan, int s, unsigned flags,
                            const void* rho_x, const void* rho_dir, int q_begin, int q_end,
                            const void* W, const double* energies, double delta, int prec,
                            void* H, void* ws, size_t ws_bytes, void* stream);

/*
 * Y = H X for nvec vectors (X, Y complex128 [nvec][dim]); H complex64 products
 * accumulated in FP32 within 16-element chunks and combined in FP64.
 */
bse_status bse_apply_H(bse_plan* plan, int s, const void* H, const void* X, void* Y, int nvec,
                       void* stream);

/*
 * A7 + A8.  Haydock recursion (Lanczos from v_0 = P/|P|, classical
 * Gram-Schmidt applied twice against the whole basis each step, FP64) and
 * eps_2(w) = -C |P|^2 Im g(w + i eta) with the continued fraction
 * g(z) = 1/(z - a_0 - b_1^2/(z - a_1 - ...)), no terminator
 * (Eq. epsilon_chi_bar in the TDA, Appendix A resolvent).
 * omega float64 [nw] (Ha), eps2 float64 [nw], ab float64 [2*nsteps]
 * (a_0..a_{n-1}, then b_0 = 0, b_1..b_{n-1}), steps_done int32 [1]: fewer than
 * nsteps after a breakdown (b_{j+1} <= 1e-6 |H v_j|, the FP32 rounding level of
 * the product), which is exact, not an error.  One persistent cooperative launch; device-side barrier waits are
 * bounded and report BSE_ERR_TIMEOUT through bse_status_read.
 */
bse_status bse_spectrum(bse_plan* plan, int s, const void* H, const void* P, int nsteps,
                        const double* omega, int nw, double eta,
                        double* eps2, double* ab, int* steps_done,
                        void* ws, size_t ws_bytes, void* stream);

/*
 * q-point symmetry (Sec. III A).  The planner finds the point group of the lattice as integer
 * matrices R on reduced reciprocal coordinates (R^T M R = M for the reciprocal metric M, mapping the
 * k mesh onto itself; symmorphic, no fractional translations), ordered identity first then by
 * ascending row-major entries, and reduces the q mesh under R and time reversal: q visited in
 * ascending index, an unassigned q becomes irreducible and every image s R q (s = +1, then -1, for
 * each R in order) not yet assigned maps to it with G0 = q - s R q_IBZ.
 * bse_symmetry (host or device plan): *nops, *nibz; ibz int32 [nq] (first nibz entries: the
 * irreducible q indices, ascending); qmap int32 [nq][6] = (irreducible index, operation, time
 * reversal, G0x, G0y, G0z); perm int32 [nq][ng_max]: position on the sphere of q_IBZ of
 * s R^-1 (g_p + G0) for each point p of the sphere of q (-1 past the sphere).  Outputs may be NULL.
 * bse_unfold_w: W complex64 [nq][ng_max][ng_max] for q in [q_begin, q_end) from W_ibz complex64
 * [nibz][ng_max][ng_max] (row i belongs to ibz[i]): W_pp'(q) = W_ibz[perm p][perm p'], conjugated
 * for time reversal (Sec. III A); entries past the sphere are zero.  Errors: BSE_ERR_ARG.
 */
bse_status bse_symmetry(const bse_plan* plan, int s, int* nops, int* nibz, int32_t* ibz, int32_t* qmap,
                        int32_t* perm);
bse_status bse_unfold_w(bse_plan* plan, int s, const void* W_ibz, void* W, int q_begin, int q_end, void* stream);

/*
 * Exciton energies and oscillator strengths from a Haydock recursion: the eigenvalues theta_i of its
 * tridiagonal T (diagonal a_j, off-diagonal b_j) and the weights w_i = (first component of the
 * normalised eigenvector)^2, the poles and residues of g(z) = sum_i w_i/(z - theta_i).  Converged Ritz
 * pairs are eigenpairs of H: E_l and |P^H A_l|^2/|P|^2 (the spectral representation of Eqs. resolvent
 * and epsilon_chi_bar); sum_i w_i = 1.
 * ab         float64 [2*nsteps] as written by bse_spectrum (a_0..a_{n-1}, then b_0 = 0, b_1..b_{n-1}).
 * steps_done int32 [1] as written by bse_spectrum; n = min(steps_done, nsteps).
 * theta      float64 [nsteps] ascending (entries >= n set to 0);  weight float64 [nsteps].
 * ws         bse_workspace_size(BSE_WS_RITZ, nsteps) bytes (any plan and system).
 * One thread per Ritz value in FP64: bisection on Sturm counts, inverse iteration with partial
 * pivoting.  No device-side waits; capturable.  Errors: BSE_ERR_ARG (nsteps outside [1, 4096]),
 * BSE_ERR_WORKSPACE.
 */
bse_status bse_ritz(const double* ab, const int* steps_done, int nsteps, double* theta, double* weight, void* ws,
                    size_t ws_bytes, void* stream);

/*
 * Exciton states (Eq. bse_eig): eigenpairs H A_l = E_l A_l.  A Lanczos tridiagonalisation of Krylov
 * dimension n from the start vector X0 (complex128 [dim], any norm): the recursion of bse_spectrum
 * (FP32 products with H, Gram-Schmidt twice against the whole stored basis, FP64 coefficients), then
 * the eigenvalues of the tridiagonal T by bisection and its eigenvectors y_l by inverse iteration
 * (FP64), and A_l = sum_j y_l(j) v_j.  With n = dim and an X0 that overlaps every eigenvector (e.g.
 * a random vector) the pairs are all eigenpairs of H; with n < dim they are the Ritz pairs of the
 * Krylov space (extreme and isolated states first).  Eigenvalues that coincide to rounding appear
 * once; a breakdown (an invariant Krylov space) ends the recursion early, with steps_done < n.
 * theta float64 [n] ascending (entries >= steps_done zero);  A complex64 [n][dim], row l the unit
 * eigenvector of theta_l (optional, may be NULL);  ab float64 [2 n] and steps_done int32 [1] as in
 * bse_spectrum.  ws: bse_workspace_size(BSE_WS_STATES, n) bytes (about n dim 16 B + 7 n^2 8 B).
 * One persistent cooperative launch (bounded grid-barrier waits, BSE_ERR_TIMEOUT through
 * bse_status_read) and two kernels.  Errors: BSE_ERR_ARG (n outside [1, dim]), BSE_ERR_WORKSPACE.
 */
bse_status bse_exciton_states(bse_plan* plan, int s, const void* H, const void* X0, int n, double* theta, void* A,
                              double* ab, int* steps_done, void* ws, size_t ws_bytes, void* stream);

/*
 * A7 + A8 for a batch of n <= 24 systems of one plan in ONE persistent cooperative
 * launch: the grid (one CTA per SM) is split into per-system CTA groups sized by each
 * system's H bytes (at least one CTA), each group runs the recursion of bse_spectrum on
 * its system with group-local bounded barriers, so small and large systems progress
 * together (the layered 2D batch of Sec. V-sized sheets).  Per-system arguments are host
 * arrays of device pointers: H[i], P[i], eps2[i] [nw], ab[i] [2*nsteps], steps_done[i],
 * ws[i] (bse_workspace_size(BSE_WS_SPECTRUM, nsteps) of that system, ws_bytes[i]).
 * All systems share nsteps, omega (device, nw) and eta.
 */
bse_status bse_spectrum_batch(bse_plan* plan, int n, const int* systems, const void* const* H,
                              const void* const* P, int nsteps, const double* omega, int nw, double eta,
                              double* const* eps2, double* const* ab, int* const* steps_done,
                              void* const* ws, const size_t* ws_bytes, void* stream);

/*
 * bse_spectrum without a caller workspace.  The paper has no counterpart: this
 * entry point exists for callers that cannot call cudaMalloc when they run the
 * spectrum - for example code behind a foreign-function boundary that is handed
 * only the input and output buffers by a host framework that owns all device
 * memory.  The scratch (Krylov basis, projection partials, barrier words) is a
 * 48 MiB file-scope device array inside the library, held on every device that
 * loads the library until the process exits; no memory is allocated by this
 * call.  Arguments and outputs are those of bse_spectrum.
 * Limit: the scratch bse_workspace_size(BSE_WS_SPECTRUM, nsteps) reports must
 * fit in 48 MiB (roughly nsteps * dim * 16 bytes + nsteps * 16 KiB); larger
 * requests return BSE_ERR_ARG with the sizes in bse_last_error().
 * Every call made outside stream capture looks up the array's device address
 * afresh (so a cudaDeviceReset between calls is harmless); a call made while its
 * stream is being captured reuses the address found by the last call outside
 * capture on that device, so make one call on each device before any capture.  Every call shares
 * the one array and it keeps the last call's contents (the words that must
 * start at zero are cleared by each call): calls that overlap on the GPU race.
 */
bse_status bse_spectrum_static(bse_plan* plan, int s, const void* H, const void* P, int nsteps,
                               const double* omega, int nw, double eta,
                               double* eps2, double* ab, int* steps_done, void* stream);

/*
 * A9.  Adjoint of L(eps_2) given dL_deps2 float64 [nw].  Recomputes the
 * Lanczos basis, forms G_H = -C sum_w g(w) i xt(w) x(w)^H from the Krylov
 * resolvent (x = R(z)P, xt = R(conj z)P), and chains it:
 *   dL_ddelta float64 [1]  = Re tr G_H,
 *   dL_dH     complex64 [dim][dim] (optional, may be NULL: then kept in ws),
 *   dL_drho_x complex64 [dim][ng_max], dL_drho_dir as rho_dir for all q,
 *   dL_dW     complex64 [nq][ng_max][ng_max],
 * each stored entry taken as a free variable; complex gradients are
 * dL/dRe + i dL/dIm.  Any of dL_drho_x, dL_drho_dir, dL_dW may be NULL.
 */
bse_status bse_spectrum_backward(bse_plan* plan, int s, const void* H, const void* P, int nsteps,
                                 const double* omega, int nw, double eta, const double* dL_deps2,
                                 const void* rho_x, const void* rho_dir, const void* W,
                                 double* dL_ddelta, void* dL_dH, void* dL_drho_x,
                                 void* dL_drho_dir, void* dL_dW,
                                 void* ws, size_t ws_bytes, void* stream);

/*
 * Tile-shape variants of the pair-density kernel (step A2) and their autotuner.
 *
 * Two routes compute the pair densities.  The plane-wave correlation kernel (variant indices 64,
 * 65 and 66, listed first with rows = 0; 65 issues the gather of the next G2 row one iteration ahead,
 * 64 does not; 66 computes the vv' and cc' products of a direct-set block in two CTAs, two per SM,
 * and is listed where that fits shared memory; all three give bit-identical results) sums conj(c_nk(G2 - G)) c_mk'(G2) over the
 * sphere of k' with a shared-memory index box of the sphere of k; it is compiled for Nv, Nc in
 * {1..3} x {1..3}, (3, 4), (4, 4) and is the default where valid.  The pruned-FFT kernels (the paper's route) are
 * compiled per real-space grid (threads per CTA, z-lines per chunk, maximum band products and
 * band slabs per CTA, sphere points per thread, vv'/cc' merged in one CTA or not); without a
 * valid correlation variant the first valid FFT variant is the default.  Both give the same
 * densities to FP32 rounding; the FFT variants among themselves bit for bit.  The real-space
 * stage (BSE_PD_REALSPACE) always runs an FFT variant of the grid and also keeps a copy of the
 * coefficients in the pair workspace for the correlation kernel.  No counterpart in the paper.
 *
 * bse_pair_variants lists the valid variants of system s (up to cap entries of out, the
 * total in *count) and the index in use (*current).  bse_set_pair_variant selects one by its
 * index (-1 restores the default); BSE_ERR_ARG if the index is not valid for the system.
 * bse_autotune_pair times every valid variant on the direct pair densities of q in
 * [q_begin, q_end) (one warm-up launch, then reps timed launches each, CUDA events on stream),
 * writes the mean milliseconds per launch to ms[i] (i < cap, in bse_pair_variants order),
 * selects the fastest and returns its index in *chosen.  It needs the pair workspace of
 * bse_pair_densities (its contents only feed the timed launches) and rho_dir with room for
 * bse_rho_dir_count(q_begin, q_end) vectors, whose contents it overwrites.  It synchronises
 * the stream (not capturable).  Errors: BSE_ERR_ARG, BSE_ERR_WORKSPACE, BSE_ERR_UNSUPPORTED,
 * BSE_ERR_CUDA (the previous selection is kept).
 */
typedef struct {
  int index;              /* variant id (argument of bse_set_pair_variant) */
  int threads;            /* threads per CTA */
  int rows;               /* z-lines per pipelined chunk; 0: the plane-wave correlation kernel */
  int max_products;       /* band products per CTA */
  int max_bands;          /* band slabs per CTA */
  int points_per_thread;  /* sphere points accumulated per thread */
  int merged;             /* 1: vv' and cc' products of a block in one CTA */
} bse_pair_variant;

bse_status bse_pair_variants(const bse_plan* plan, int s, bse_pair_variant* out, int cap, int* count,
                             int* current);
bse_status bse_set_pair_variant(bse_plan* plan, int s, int index);
bse_status bse_autotune_pair(bse_plan* plan, int s, void* ws, size_t ws_bytes, void* rho_dir, int q_begin,
                             int q_end, int reps, float* ms, int cap, int* chosen, void* stream);

/*
 * Static RPA screening from the system's own states (Sec. II A-B, Eqs. chi0_GG and
 * epsilon_-1; the W_GG'(q) form of Sec. III A).  Produces the W that bse_build_kernel takes,
 * for q in [q_begin, q_end):
 *   chi0_GG'(q) = 4/(Omega Nk) sum_{k,v,c} rho(G) conj(rho(G')) / (e_vk - e_c,k+q),
 *   rho = rho_vc^{k,k+q}(G) (bse_pair_densities with BSE_PD_CHI0), bare energies with the
 *   system's gap floor; eps = 1 - v^1/2 chi0 v^1/2 (v^1/2 = sqrt(4 pi)/|q+G|); at q = 0 the
 *   G = 0 row and column from the k.p dipole P (bse_pair_densities, BSE_PD_EXCHANGE);
 *   eps^-1 by `iterations` Newton-Schulz steps from 2/(1 + R) I (R: Gershgorin bound);
 *   W = v^1/2 eps^-1 v^1/2, at q = 0 head [eps^-1]_00 12 pi/q_c^2 (q_c^3 = 6 pi^2/(Omega Nk))
 *   and zero wings.
 * rho_chi  complex64 [(q_end - q_begin) Nk Nv Nc][ng_max] from BSE_PD_CHI0 for the same range;
 *          overwritten with the scaled pair vectors.
 * energies float64 [Nk][Nb];  P complex128 [dim] (needed when q_begin = 0).
 * W        complex64 [Nq][ng_max][ng_max]; the rows of q in the range are written (zero padded).
 * residual float32 [q_end - q_begin] on the device (optional): max |I - eps X| per q.
 * ws       bse_workspace_size(BSE_WS_SCREEN, q_end - q_begin) bytes.
 * Errors: BSE_ERR_ARG, BSE_ERR_WORKSPACE, BSE_ERR_UNSUPPORTED (slab Coulomb).
 */
bse_status bse_screening(bse_plan* plan, int s, void* rho_chi, const double* energies, const void* P, int q_begin,
                         int q_end, int iterations, void* W, float* residual, void* ws, size_t ws_bytes,
                         void* stream);

/*
 * The BSE beyond the Tamm-Dancoff approximation (Appendix A): e-h pairs S = (k, v, c) coupled to
 * h-e pairs (k, c -> v).  In the basis (e-h, h-e) the Hamiltonian is
 *   H2 = [[A, B], [-conj(B), -conj(A)]],
 * A the Tamm-Dancoff H of bse_build_kernel, B the coupling block below.
 *
 * Number of complex vectors of rho_cpl for q in [q_begin, q_end) (each ng_max long):
 * 2 Nv Nc per upper block.
 */
bse_status bse_rho_cpl_count(const bse_plan* plan, int s, int q_begin, int q_end, long long* nvec);

/*
 * Coupling block B = 2 Bx - Bd (Eqs. V_eh and W_SS with the band labels of the h-e pair):
 *   Bx_SS' = 1/(Omega Nk) sum_{G != 0} conj(rho_vc^{kk}(G)) vbar(G) conj(rho_v'c'^{k'k'}(-G)),
 *   Bd_SS' = 1/(Omega Nk) sum_{G,G'} conj(rho_vc'^{kk'}(G)) W_GG'(k'-k) rho_cv'^{kk'}(G').
 * B is symmetric (B^T = B) for W with the reciprocity W_{-G,-G'}(-q) = conj(W_GG'(q)).
 * rho_x    as in bse_pair_densities (BSE_PD_EXCHANGE).
 * rho_cpl  complex64 [nvec][ng_max] from bse_pair_densities with BSE_PD_COUPLING (rho_dir
 *          argument) for the same q range: per q, nblk_q Nv Nc vectors rho~_vc'^{kk'}
 *          (block-major, then v, c'), then nblk_q Nc Nv vectors rho~_cv'^{kk'} (block-major,
 *          then c, v'), with the G = g_p(q) - G0 convention of rho_dir.
 * BSE_BC_INIT writes 2 Bx on the upper block triangle (k <= k'); BSE_BC_DIRECT subtracts Bd for
 * the upper blocks of q in [q_begin, q_end) and writes the mirror B_k'k = B_kk'^T (diagonal blocks
 * (B + B^T)/2); BSE_BC_MIRROR (not with DIRECT) completes an INIT-only build the same way.
 * Bm       complex64 [dim][dim] row-major.  W, prec as in bse_build_kernel.
 * ws       bse_workspace_size(BSE_WS_COUPLING, q_end - q_begin) bytes (0 for INIT alone).
 * Errors: BSE_ERR_ARG, BSE_ERR_WORKSPACE, BSE_ERR_UNSUPPORTED (Nv Nc > 16, or a q = 0 sphere
 * without its -G partners).
 */
bse_status bse_build_coupling(bse_plan* plan, int s, unsigned flags, const void* rho_x, const void* rho_cpl,
                              int q_begin, int q_end, const void* W, int prec, void* Bm, void* ws, size_t ws_bytes,
                              void* stream);

/*
 * eps_2 of the coupled problem (Eqs. Dyson_eh_rearrange and epsilon_chi_bar with f = diag(1, -1)):
 *   eps_2(w) = -C Im[Pt^H (z - H2)^{-1} F Pt],  Pt = (P, -conj P),  F = diag(1, -1),  z = w + i eta,
 * the h-e optical element being -conj(P).  Evaluated by Lanczos on H2 in the inner product of
 * M = F H2 (Hermitian; positive definite for a stable system) from s = F Pt, which gives
 *   eps_2 = -C b_0^2 Im[g(z)/z],  g(z) = 1/(z - b_1^2/(z - b_2^2/(...))),  b_0 = |s|_M;
 * the diagonal coefficients vanish by the e-h / h-e symmetry, and the recursion runs on the e-h
 * halves of the Lanczos vectors (one product with A and one with B per step; full
 * reorthogonalisation, twice, against the vectors of the same parity).
 * A, Bm    complex64 [dim][dim] (A Hermitian, Bm symmetric; full matrices).
 * P        complex128 [dim].  omega float64 [nw] (Ha).  nsteps in [1, 2 dim].
 * eps2     float64 [nw];  b float64 [nsteps]: b_0 = |s|_M, b_1..b_{n-1};  steps_done int32 [1]:
 *          fewer than nsteps after a breakdown (|w_j|_M <= 1e-6 |H2 q_{j-1}|_M), not an error.
 * ws       bse_workspace_size(BSE_WS_COUPLED, nsteps) bytes.
 * A negative squared M-norm (M not positive definite), or P = 0, stops the recursion and sets
 * BSE_ERR_INDEFINITE in the plan's status word (read with bse_status_read).  4 kernels per step,
 * no device-side waits; capturable in a CUDA graph.
 * Errors: BSE_ERR_ARG, BSE_ERR_WORKSPACE, BSE_ERR_UNSUPPORTED (dim > 65536).
 */
bse_status bse_spectrum_coupled(bse_plan* plan, int s, const void* A, const void* Bm, const void* P, int nsteps,
                                const double* omega, int nw, double eta, double* eps2, double* b, int* steps_done,
                                void* ws, size_t ws_bytes, void* stream);

/*
 * Macroscopic dielectric function from TDDFT with local fields (Sec. II A-B: Eqs. epsilon_M,
 * epsilon_-1, Dyson_GG, chi0_GG) in the optical limit q -> 0 along qhat, on the q = 0 sphere
 * (ng0 vectors G).  Bulk (3D Coulomb) systems with a q = 0 sphere symmetric under G -> -G.
 *
 * bse_chi0_optical: the symmetrised Adler-Wiser response chi~0 = v^1/2 chi0 v^1/2 for nw frequencies,
 *   chi~0_GG'(w) = 2/(Omega Nk) sum_S [ a_S(G) conj a_S(G') / (w - de_S + i eta)
 *                                      - abar_S(G) conj abar_S(G') / (w + de_S + i eta) ],
 *   a_S(G) = v^1/2(G) rho_vc^{kk}(G), abar_S(G) = v^1/2(G) conj(rho_vc^{kk}(-G)) for G != 0 (v^1/2(G) =
 *   sqrt(4 pi)/|G|), a_S(0) = sqrt(4 pi) conj(P_S), abar_S(0) = -sqrt(4 pi) P_S (the k.p limit of
 *   Eq. density_matrix), de_S = e_c + delta - e_v (delta = 0: the band energies as given).
 *   rho_x    complex64 [dim][ng_max] and P complex128 [dim] from bse_pair_densities (EXCHANGE).
 *   energies float64 [Nk][Nb];  omega float64 [nw] (Ha);  eta > 0 (Ha).
 *   chi0     complex64 [nw][ng0][ng0] row-major (row G, column G').
 *   ws       bse_workspace_size(BSE_WS_CHI0) bytes.
 *   FP32 products and sums (64 x 64 output tiles per frequency).
 * bse_xc_kernel_alda: F = v^-1/2 f_xc v^-1/2 of the adiabatic local-density kernel,
 *   F_GG' = |G| f_xc(G - G') |G'| / (4 pi),  f_xc(G) = (1/N_r) sum_r f_xc(r) exp(-iG.r),
 *   f_xc(r) = d^2(n eps_xc)/dn^2 at n(r) = 2/(Omega Nk) sum_{k,v} |u_vk(r)|^2 (floor 1e-6 bohr^-3), eps_xc
 *   Slater exchange + Perdew-Zunger (Ceperley-Alder) correlation, spin-unpolarised; row and column
 *   G = 0 are zero (q -> 0).  pair_ws: the pair workspace after bse_pair_densities(BSE_PD_REALSPACE)
 *   (it holds u_nk(r) on the grid).  F complex64 [ng0][ng0].  ws: bse_workspace_size(BSE_WS_ALDA).
 *   Errors: BSE_ERR_UNSUPPORTED when the grid cannot hold the G - G' box of the sphere.
 * bse_epsilon_macro: for every frequency, eps^-1 = I + (I - chi~0 (I + F))^-1 chi~0 and
 *   eps_M(w) = 1/[eps^-1]_00 (F = NULL: the RPA, K = v).  One Dyson system per frequency, solved by
 *   Gaussian elimination with partial pivoting in FP32 (one CTA per frequency); eps_m complex128 [nw].
 *   ws: bse_workspace_size(BSE_WS_EPSM, nw).  Errors: BSE_ERR_UNSUPPORTED for ng0 > 4096.
 * Inputs are scanned for NaN/Inf (BSE_ERR_NONFINITE through bse_status_read).  No device-side waits.
 */
bse_status bse_chi0_optical(bse_plan* plan, int s, const void* rho_x, const void* P, const double* energies,
                            double delta, const double* omega, int nw, double eta, void* chi0, void* ws,
                            size_t ws_bytes, void* stream);
bse_status bse_xc_kernel_alda(bse_plan* plan, int s, const void* pair_ws, size_t pair_ws_bytes, void* F, void* ws,
                              size_t ws_bytes, void* stream);
bse_status bse_epsilon_macro(bse_plan* plan, int s, const void* chi0, const void* F, int nw, void* eps_m, void* ws,
                             size_t ws_bytes, void* stream);

/*
 * Failure injection: limit (ns) of every grid-barrier wait of the spectrum kernels (steps A7,
 * A8 and their recomputation in the adjoint) on the current device; default 2e9.  A wait that
 * exceeds it sets BSE_ERR_TIMEOUT in the plan's status word and the kernel returns; with 0
 * every wait gives up at once, which exercises that path without a fault or a hang.  The
 * other kernels' waits keep their fixed 2 s limit.  Synchronous; not capturable.  No
 * counterpart in the paper.  Errors: BSE_ERR_CUDA.
 */
bse_status bse_set_wait_limit(unsigned long long ns);

/* Synchronise the stream and return (then clear) the plan's device status word. */
bse_status bse_status_read(bse_plan* plan, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* BSE_H */
