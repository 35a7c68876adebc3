// Internal declarations shared by the host planner, the C-ABI glue and the CUDA kernels.
#pragma once

#include <array>
#include <cstdint>
#include <vector_types.h>
#include <string>
#include <vector>

#include "bse.h"

namespace bse {

constexpr double kPi = 3.141592653589793;

// Device-side description of one system: pointers into the plan's device tables.
struct DevSys {
  int nkpt, nb, nv, nc, dim, npw_max, ng_max, ng0, nq;
  int n1, n2, n3;                 // FFT grid
  int nk1, nk2, nk3;              // k mesh
  int fwf[3], fpair[3];           // max |g| per axis of wavefunction / pair spheres (after G0)
  double norm, prefactor, omega_cell;
  const char4* gk;                // [nkpt][npw_max]  (g1,g2,g3,0) of the k spheres
  const int* npw;                 // [nkpt]
  const char4* gq;                // [nq][ng_max]      (g1,g2,g3,0) of the q spheres
  const int* ngq;                 // [nq]
  const int4* blocks;             // [nblocks] (ik, ik2, iq, g0 packed as (g0+1) bits)
  const long long* qblk_off;      // [nq+1] first block of each q (blocks sorted by q, then ik)
  const long long* qvec_off;      // [nq+1] first rho_dir vector of each q
  const int* blkidx;              // [nq][nkpt] global block of (q, k) with k <= k + q, else -1
  const double* kgq;              // [nkpt][npw_max] qhat.(k+G), Cartesian
  const float* xscale;            // [ng_max] sqrt(2 vbar(G) / (Omega Nk)), 0 at G = 0 and beyond ng0
  const float* vsq;               // [nq][ng_max] sqrt(4 pi)/|q+G| (0 at q+G = 0 and beyond ngq)
  long long nblocks;
  int pair_variant;               // index of the pair-kernel variant chosen for this system, -1 = first valid
  const int* gminus0;             // [ng0] index of -G on the q = 0 sphere (-1 if absent)
  const int* qperm;               // [nq][ng_max] sphere map of q onto its irreducible point (-1 padded)
  const int2* qsym;               // [nq] (irreducible index, time reversal)
  int nibz;
  // k-point symmetry: the upper blocks that are not representatives, (ik, ik2, rep ik, rep ik2), the last
  // stored as -(rep ik2 + 1) when the block is the representative's Hermitian mirror
  const int4* fill;
  long long nfill;
  // Tensor-core direct densities (tcpair.cu).  The k' mesh is cut into regions of tc_rg[0] x tc_rg[1] x
  // tc_rg[2] points (tc_nr regions per axis, tc_rsize points each); region r has a K layout, the union of
  // the spheres of its k' in lexicographic order (tc_kcount[r] entries, padded to tc_kpad).
  int tc_rg[3], tc_nr[3], tc_nreg, tc_rsize, tc_kpad;
  const char4* tc_klist;          // [tc_nreg][tc_kpad] G of each K position
  const int* tc_kcount;           // [tc_nreg]
  const short* tc_kpos;           // [nkpt][npw_max] K position of sphere point i of k in its region's layout
  const short* tc_pmap;           // [nq][(2 fwf0 + 1)(2 fwf1 + 1)(2 fwf2 + 1)] sphere position of g on q, -1 if absent
};

struct SysPlan {
  bse_system sys;
  std::vector<int4> fill;                      // host copy of DevSys::fill
  DevSys d;                       // device view (pointers valid on the plan's device)
  std::vector<std::vector<int32_t>> gk, gq;   // host spheres, flattened (g1,g2,g3)*
  std::vector<int32_t> blocks;                 // host (ik, ik2, iq, g0x, g0y, g0z) per block
  std::vector<long long> qblk_off, qvec_off;
  bool gminus0_complete = false;  // every G of the q = 0 sphere has -G on it
  // q-point symmetry (Sec. III A): operations (row-major integer 3x3 on reduced reciprocal
  // coordinates), irreducible q points, per q (iq_ibz index, op, tr, G0x, G0y, G0z), sphere maps
  std::vector<std::array<int, 9>> ops;
  std::vector<int> ibz, qmap, qperm;
  void* dmem = nullptr;           // one device allocation holding every table
};

}  // namespace bse

struct bse_plan {
  int device = 0;
  std::vector<bse::SysPlan> sys;
  int* d_status = nullptr;        // device status word (bse_status of the first device-side error)
};

namespace bse {
bse_status set_error(bse_status st, const std::string& msg);
bse_status cuda_check(int err, const char* what);

// Kernel launchers (defined in the .cu files); all return cudaError_t as int.
int launch_realspace(const DevSys& d, const void* coef, void* u, void* stream);
int launch_pair_exchange(const DevSys& d, const void* u, void* rho_x, int* status, void* stream);
int launch_pair_direct(const DevSys& d, const void* u, void* rho_dir, int q_begin, int q_end, long long vbase,
                       int* status, void* stream);
int launch_dipole(const DevSys& d, const void* coef, const double* energies, double gap_floor, void* P, void* stream);
int launch_pair_chi0(const DevSys& d, const void* u, void* rho, int q_begin, int q_end, int* status, void* stream);
size_t screen_ws_bytes(const DevSys& d, long long qchunk);
int launch_screening(const DevSys& d, void* rho_chi, const double* energies, const void* P, int q_begin, int q_end,
                     int iterations, void* W, float* residual, void* ws, double gap_floor, void* stream);
int pair_supported(const DevSys& d);
size_t pair_ws_bytes(const DevSys& d);
int gcorr_valid(const DevSys& d);
int tcpair_valid(const DevSys& d);
size_t tcpair_ws_bytes(const DevSys& d);
int launch_tcpair(const DevSys& d, const void* coef, void* ws, void* rho_dir, int q_begin, int q_end,
                  long long vbase, int* status, void* stream);
int launch_pair_direct_tensor(const DevSys& d, void* ws, void* rho_dir, int q_begin, int q_end, long long vbase,
                              int* status, void* stream);
int gcorr_split_valid(const DevSys& d);
int gcorr_threads(const DevSys& d);
int launch_gcorr(const DevSys& d, const void* coef, void* out, int kind, int mode, int q0, int nqc, long long vbase,
                 long long cells, int pf, void* stream);
// Pair-kernel variants compiled for this system: writes up to cap (index, threads, rows, pmax, bmax, ppt,
// merged) septets, returns the number valid; pair_variant_current returns the index pick() uses.
int pair_variants(const DevSys& d, int* out, int cap);
int pair_variant_current(const DevSys& d);

int launch_kernel_init(const DevSys& d, const void* rho_x, const double* energies, double delta, void* H, void* stream);
size_t gram_ws_bytes(const DevSys& d);
int launch_kernel_init_tc(const DevSys& d, const void* rho_x, const double* energies, double delta, void* H,
                          void* ws, int* status, void* stream);
int launch_mirror(const DevSys& d, void* H, void* stream);
int launch_symfill(const DevSys& d, void* H, void* stream);
int launch_kernel_direct_range(const DevSys& d, const void* rho_dir, int q_begin, int q_end, long long b_begin,
                               long long b_count, long long vbase, long long max_rows, const void* W, int prec,
                               void* H, void* ws, int* status, void* stream);
int launch_gemm_wr_tc(const DevSys& d, const void* rho_dir, int q_begin, int q_end, long long vbase,
                      long long max_rows, const void* W, void* X, void* split_ws, int side_c, int* status,
                      void* stream);
size_t tc_split_bytes(const DevSys& d, long long qchunk, long long w);
// Coupling block B of the BSE beyond the Tamm-Dancoff approximation (build.cu, coupled.cu).
int launch_pair_coupling(const DevSys& d, const void* u, void* rho_cpl, int q_begin, int q_end, long long vbase,
                         int* status, void* stream);
size_t coupling_ws_bytes(const DevSys& d, long long qchunk);
int launch_coupling_init(const DevSys& d, const void* rho_x, void* Bm, void* ws, void* stream);
int launch_coupling_direct_range(const DevSys& d, const void* rho_cpl, int q_begin, int q_end, long long b_count,
                                 long long vbase, long long max_rows, const void* W, int prec, void* Bm, void* ws,
                                 int* status, void* stream);
int launch_coupling_mirror(const DevSys& d, void* Bm, void* stream);
size_t coupled_ws_bytes(const DevSys& d, long long nsteps);
size_t ritz_ws_bytes(long long nsteps);
int launch_unfold_w(const DevSys& d, const void* W_ibz, void* W, int q_begin, int q_end, void* stream);
int launch_ritz(const double* ab, const int* steps_done, int nsteps, double* theta, double* weight, void* ws,
                void* stream);
int launch_ritz_vectors(const double* ab, const int* steps_done, int nsteps, double* theta, double* weight, void* ws,
                        double* vecs, void* stream);
size_t states_ws_bytes(const DevSys& d, long long n);
int launch_exciton_states(const DevSys& d, const void* H, const void* X0, int n, double* theta, void* A, double* ab,
                          int* steps_done, void* ws, int* status, void* stream);
int launch_spectrum_coupled(const DevSys& d, const void* A, const void* Bm, const void* P, int nsteps,
                            const double* omega, int nw, double eta, double* eps2, double* b, int* steps_done,
                            void* ws, int* status, void* stream);
size_t kernel_ws_bytes(const DevSys& d, long long qchunk);
int launch_gemm_wr(const DevSys& d, const void* rho_dir, int q_begin, int q_end, long long vbase, long long max_rows,
                   const void* W, void* X, int side_c, void* stream);

// Streams n elements of elem_bytes (4: float / complex64 parts, 8: double) through a NaN/Inf check;
// a hit sets BSE_ERR_NONFINITE in *status.  n <= 0 launches nothing.
int launch_nonfinite_scan(const void* p, long long n, int elem_bytes, int* status, void* stream);

// Macroscopic dielectric function from TDDFT with local fields (tddft.cu).
size_t chi0_ws_bytes(const DevSys& d);
int launch_chi0_optical(const DevSys& d, const void* rho_x, const void* P, const double* energies, double delta,
                        const double* omega, int nw, double eta, void* chi0, void* ws, void* stream);
size_t alda_ws_bytes(const DevSys& d);
int launch_alda_kernel(const DevSys& d, const void* pair_ws, const int* m, void* F, void* ws, void* stream);
size_t epsm_ws_bytes(const DevSys& d, long long nw);
int launch_epsilon_macro(const DevSys& d, const void* chi0, const void* F, int nw, void* eps_m, void* ws,
                         void* stream);

size_t spectrum_static_capacity();
int set_wait_limit(unsigned long long ns);
int launch_spectrum_static(const DevSys& d, const void* H, const void* P, int nsteps, const double* omega, int nw,
                           double eta, double* eps2, double* ab, int* steps_done, int* status, void* stream);
int launch_apply_h(const DevSys& d, const void* H, const void* X, void* Y, int nvec, void* stream);
size_t spectrum_ws_bytes(const DevSys& d, long long nsteps);
int launch_spectrum(const DevSys& d, const void* H, const void* P, int nsteps, const double* omega, int nw,
                    double eta, double* eps2, double* ab, int* steps_done, void* ws, int* status, void* stream);
size_t backward_ws_bytes(const DevSys& d, long long nsteps);
int launch_backward(const DevSys& d, const long long* h_qblk_off, const long long* h_qvec_off, const void* H,
                    const void* P, int nsteps, const double* omega, int nw, double eta, const double* dL,
                    const void* rho_x, const void* rho_dir, const void* W, double* d_delta, void* dH, void* drho_x,
                    void* drho_dir, void* dW, void* ws, int* status, void* stream);
int upload_twiddles();
struct HayJob {
  const DevSys* d;
  const void* H;
  const void* P;
  double* eps2;
  double* ab;
  int* steps_done;
  void* ws;
};
int run_haydock_batch(const HayJob* jobs, int n, int nsteps, const double* omega, int nw, double eta, int* status,
                      void* stream);
int run_haydock(const DevSys& d, const void* H, const void* P, int nsteps, const double* omega, int nw, double eta,
                double* eps2, double* ab, int* steps_done, void* ws, int* status, void* stream, float4** V_out);
}  // namespace bse
