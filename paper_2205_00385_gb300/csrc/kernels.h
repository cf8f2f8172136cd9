// Host launchers of the library's kernels (runtime-dispatched templates).
#pragma once

#include "topo_internal.cuh"

namespace topo {

// arithmetic / storage types; T_DF = float64 storage with double-float
// arithmetic on the FP32 pipe (finest 3D grid only)
// Arithmetic / storage codes.  T_DF: double-float arithmetic (float64
// storage or pairs); T_D2: storage as double-float pairs float2 {hi, lo}.
enum { T_F64 = 0, T_F32 = 1, T_DF = 2, T_D2 = 3 };
enum { EPI_APPLY = 0, EPI_RESID = 1, EPI_SMOOTH = 2 };

// Stiffness operator of one grid level,
//   y = M (sum_e A_e^T Ke_e A_e) M x + dfix (I - M) x      (EPI_APPLY)
//   y = b - (that)                                         (EPI_RESID)
//   y = x + omega * dinv * (b - that)                      (EPI_SMOOTH)
// with Ke_e = coef_e * KE on the finest level (explicit = false) or the
// stored Galerkin element matrix Kc_e on coarse levels (explicit = true).
// Explicit levels are applied from their assembled stencil S (fixed rows
// stored as identity rows, so dfix must be 1); the element matrices Kc are
// packed upper triangles, Kc[e*tri_len(ND) + tri_idx(r, c, ND)], r <= c.
struct ApplyArgs {
  int dim;
  GridP g;
  const uint8_t* mask;
  int tc;              // arithmetic type (T_F64 / T_F32)
  int tx, ty;          // storage types of x (and b) and of y
  bool expl;
  const void* coef;    // [nel] of type tc (fine level)
  const void* Kc;      // [tri_len(ND)*nel] of type tc (coarse levels)
  const void* ke;      // host pointer to the ND*ND element matrix of type tc
  const void* wht;     // host pointer to the 8x3x3 Walsh-Hadamard blocks of KE
                       // (type tc; 3D finest grid only, else null)
  bool gal1;           // 3D level 1 without stored matrices: coef holds the
  GridP gf;            // finest-grid moduli, gf the finest grid
  const void* x;
  void* y;
  const void* b;
  const void* dinv;    // [n] of type tc
  double omega, dfix;
  int epi;
  const void* S;       // explicit levels: assembled stencil coefficients (type tc)
  const uint8_t* colfix = nullptr;   // per node column (i, j): 1 if any DOF of the
                                     // column is fixed (null: mask every node)
  int zsplit = 0;      // layers per z-chunk of the column-streaming 3D kernels, set
                       // by the autotuner (0: the launcher's occupancy heuristic)
  int variant = 0;     // float32 pair kernel: bit 0 the tile variant (0: 8-row
                       // tiles, 1: 16-row tiles), bit 1 the work-list launch (with
                       // wl set); autotuned or set by an option
  unsigned* wl = nullptr;         // the pair kernel's work-list counters (two, zero
                                  // between launches), device
  bool use_tc = false;            // float32 finest grid: the tensor-core operator
  const void* bmat = nullptr;     // its B operand (tc_pack_b), device
  int* status = nullptr;          // device word receiving TO_E_TIMEOUT from bounded waits
  Springs springs;                // finest 2D grid: springs to ground added to K (none: n = 0)
  bool clean_inputs = false;      // x zero on every fixed DOF (the solver's own vectors): the
                                  // float32 pair kernel then masks only the fixed rows' outputs
};
cudaError_t launch_apply(const ApplyArgs& a, cudaStream_t s);

// The coarse end of the V-cycle in one cluster launch (kernels_vfuse.cu):
// restriction into level l0 (from level l0 - 1's residual r), the residual
// and restriction of every level down to the coarsest, its exact solve with
// the stored inverse, then interpolation and post-smoothing back up to level
// l0 (result in lv[l0].z2).  Levels l0 .. L-1 must be stored (stencil)
// levels.  Bit for bit the same as the one-kernel-per-step sequence.
constexpr int VF_MAXL = 12;
// a level joins the fused stretch when its assembled stencil is at most this
// large (the cluster's 8-16 SMs stream it in a few microseconds)
constexpr double VF_MAX_STENCIL_BYTES = 6.0e6;
struct VFLevel {
  GridP g;
  const uint8_t* mask;
  const void* S;       // assembled stencil (levels >= l0)
  const void* dinv;
  void* b;             // right-hand side
  void* z;             // iterate (pre-smoothed, then corrected)
  void* z2;            // post-smoothed result
  void* r;             // residual
};
struct VFuseArgs {
  int l0, L;
  VFLevel lv[VF_MAXL];   // indexed by level; lv[l0 - 1] supplies the input residual
  const void* Ainv;      // coarsest inverse, type ta
  int nc;
  double omega;
};
// cluster size the fused kernel launches with on this device (0: unavailable)
int vcycle_coarse_cluster(int dim, int t, int ta);
cudaError_t launch_vcycle_coarse(int dim, int t, int ta, const VFuseArgs& a, cudaStream_t s);
// Float32 3D finest-grid operator, two element columns per thread with packed
// f32x2 arithmetic (kernels_pair.cu); pair_apply_ok tells whether it applies.
bool pair_apply_ok(const ApplyArgs& a);
cudaError_t launch_apply_pair(const ApplyArgs& a, cudaStream_t s);
// caches the pair kernel's resident-block counts for the current device
void pair_prepare();
// Float32 3D finest-grid operator on the tensor cores (kernels_tc.cu):
// B operand packing (host, 2 x 1024 floats from the float64 KE), set-up of
// the kernels' shared-memory limit (outside stream capture), applicability
// and launch.
void tc_pack_b(const double* KE, float* out);
cudaError_t tc_prepare();
bool tc_apply_ok(const ApplyArgs& a);
cudaError_t launch_apply_tc(const ApplyArgs& a, cudaStream_t s);
// occupancy queries of the level-1 Galerkin column kernel (call at set-up)
void col_prepare();
// occupancy queries of the pair-storage double-float operator (call at set-up)
void df_prepare();
// colfix[i + nnx j] = 1 if any node (i, j, k) of the grid has a fixed DOF
cudaError_t launch_colfix(const GridP& g, const uint8_t* mask, uint8_t* colfix, cudaStream_t s);
// Double-float finest-grid operator (kernels_df.cu): float64 x/b/y, float64
// moduli in coef, float64 Walsh blocks in wht; EPI_APPLY or EPI_RESID.
cudaError_t launch_apply_df(const ApplyArgs& a, cudaStream_t s);
// true if the Walsh blocks have the structural zeros (wht_zero) to rounding
bool df_blocks_ok(const double* wht64);
// Host: the eight 3x3 blocks of the hex8 KE in the corner Walsh-Hadamard basis
void wht_blocks(const double* KE, double* out64);
// Host: store the verified structural zeros exactly and round to float32
void wht_blocks_pin_zeros(double* w64, float* w32);

// dinv = 1 / diag(A) (1 on fixed DOFs)
cudaError_t launch_diag(int dim, const GridP& g, const uint8_t* mask, int tc, bool expl,
                        const void* coef, const void* Kc, const void* ke, void* dinv,
                        cudaStream_t s, const Springs& sp = Springs());

// ---- multigrid transfer and Galerkin operators (kernels_mg.cu) ----
// b_c = Pm^T r_f; when zc is not null also the coarse level's smoothing from
// a zero guess, zc = omega * dinvc * b_c.  clean: r_f is zero on every fixed
// DOF (the fine masks are then not read; same result)
cudaError_t launch_restrict(int dim, int t, const GridP& gf, const uint8_t* maskf,
                            const GridP& gc, const uint8_t* maskc, const void* rf, void* bc,
                            const void* dinvc, double omega, void* zc, bool clean,
                            cudaStream_t s);
cudaError_t launch_prolong_add(int dim, int t, const GridP& gf, const uint8_t* maskf,
                               const GridP& gc, const void* zc, void* zf, cudaStream_t s);
// z = omega * dinv * b (smoothing from a zero initial guess); if bout != 0 the
// input (of type tin) is also converted into bout (type t).
cudaError_t launch_presmooth(int t, int tin, long long n, const void* bin, void* bout,
                             const void* dinv, double omega, void* z, cudaStream_t s);
cudaError_t launch_galerkin_fine(int dim, int t, const GridP& gc, const GridP& gf,
                                 const void* coef, const void* Qc, void* Kc, cudaStream_t s);
cudaError_t launch_galerkin_coarse(int dim, int t, const GridP& gc, const GridP& gf,
                                   const void* Kf, void* Kc, cudaStream_t s);
// 3D level 1 kept implicit: its diagonal from the finest moduli (qdiag: host
// table [8 children][8 corners][3] of diag(Q_ch)), and level-2 element
// matrices from the finest moduli with 64 tables R (device, [64][576]).
cudaError_t launch_diag_l1(int t, const GridP& g1, const GridP& gf, const uint8_t* mask,
                           const double* qdiag, const void* coef, void* dinv, cudaStream_t s);
cudaError_t launch_galerkin_l2(int t, const GridP& g2, const GridP& gf, const void* coef,
                               const void* R, void* Kc, cudaStream_t s);
// Assembled stencil of a stored level (16-byte coefficient groups, fixed
// rows as identity rows, fixed columns zero) from its packed element
// matrices; stencil_values gives its length in values of type t.
cudaError_t launch_stencil_assemble(int dim, int t, const GridP& g, const uint8_t* mask,
                                    const void* Kc, void* S, cudaStream_t s);
long long stencil_values(int dim, int t, const GridP& g);
// coarsest grid: the dense matrix A (float64, row-major) from the level's
// packed element matrices of storage t; its Cholesky-based explicit inverse
// (float64); y = A x with A float64 and x, y of storage t
cudaError_t launch_dense_assemble(int dim, int t, int ta, const GridP& g, const uint8_t* mask,
                                  const void* Kc, void* A, double shift, cudaStream_t s);
cudaError_t launch_cholesky_inverse(int t, int n, void* A, void* Ainv, int* status,
                                    cudaStream_t s);
cudaError_t launch_dense_gemv(int ta, int t, int n, const void* A, const void* x, void* y,
                              cudaStream_t s);
cudaError_t launch_convert(int tin, int tout, long long n, const void* in, void* out,
                           cudaStream_t s);

// ---- vector kernels (kernels_blas.cu) ----
cudaError_t launch_dot(long long n, const double* a, const double* b, double* partials,
                       unsigned* counter, double* out, cudaStream_t s);
// alpha = scal[num] / scal[den]; x += alpha p; r -= alpha q; scal[rr] = r.r
cudaError_t launch_cg_xr(long long n, double* x, double* r, const double* p, const double* q,
                         double* scal, int num, int den, int rr, double* partials,
                         unsigned* counter, cudaStream_t s, double* host_rr = nullptr);
// beta = scal[num] / scal[den]; p = z + beta p
cudaError_t launch_cg_p(long long n, double* p, const double* z, const double* scal, int num,
                        int den, cudaStream_t s);
cudaError_t launch_copy(long long n, const double* a, double* b, cudaStream_t s);
cudaError_t launch_scale_by_inv_sqrt(long long n, double* a, const double* s2, cudaStream_t s);
// ---- float64-accurate long vectors (kernels_vec.cu) ----
// Storage: V_F64 = float64 with float64 arithmetic (FP64 path); V_DF2 =
// float2 {hi, lo} double-float pairs with double-float arithmetic on the
// FP32 pipe (mixed path), 8 bytes per entry either way.
enum VecT { V_F64 = 0, V_DF2 = 1 };
cudaError_t launch_vdot(long long n, int vt, const void* a, const void* b, double* partials,
                        unsigned* counter, double* out, cudaStream_t s);
// out = in with a change of storage (split, widen or copy)
cudaError_t launch_vconvert(long long n, int tin, const void* in, int tout, void* out,
                            cudaStream_t s);
// x = 0 on the fixed DOFs (mask per node, bit c for DOF c), storage vt
cudaError_t launch_zero_fixed(long long nn, int dim, const uint8_t* mask, int vt, void* x,
                              cudaStream_t s);
// a *= 1/sqrt(*s2)
cudaError_t launch_vscale_inv_sqrt(long long n, int vt, void* a, const double* s2,
                                   cudaStream_t s);
// G[i + ldg*j] = sum_k A[k + i*n] B[k + j*n], i < na (na_dev overrides when
// non-null), j < nb (likewise); one pass over the data; one counter
cudaError_t launch_gram(long long n, int vt, const void* A, int na, const int* na_dev,
                        const void* B, int nb, const int* nb_dev, double* G, int ldg,
                        double* partials, unsigned* counter, cudaStream_t s);
// G = A^T B for a product known to be symmetric (A^T K A with B = K A): the
// upper triangle is summed (about half the tiles) and mirrored
cudaError_t launch_gram_sym(long long n, int vt, const void* A, const void* B, int m, double* G,
                            int ldg, double* partials, unsigned* counter, cudaStream_t s);
// y = beta*y + sign * sum_i c[i] A[:, i] (i < m, or *m_dev); if rr != 0 also
// writes |y - w|^2 (w may be null) to *rr.  A and w have storage vt, y has
// storage yt (yt = vt, or V_F64 with vt = V_DF2).
// y <- y - A c (m = *m_dev columns when given) and then h = A^T y for the
// updated y, in one pass over A (a Gram-Schmidt pass fused with the next
// pass's projections); m <= 12
cudaError_t launch_combine_dots(long long n, int vt, const void* A, int m, const int* m_dev,
                                const double* c, void* y, double* h, double* partials,
                                unsigned* counter, cudaStream_t s);
cudaError_t launch_combine(long long n, int vt, const void* A, int m, const int* m_dev,
                           const double* c, double sign, double beta, void* y, int yt,
                           const void* w, double* rr, double* partials, unsigned* counter,
                           cudaStream_t s);
// Gram-Schmidt step of the QR factorisation of the CARM basis: column src
// of R (norm^2 before in scal[n0], after in scal[n1]) is appended to the
// orthonormal factor at position ints[I_KCOUNT] if it kept more than tol of
// its length, normalised; column src of the triangular factor Rt (ld MAXB)
// receives its projections h1 + h2 on the earlier columns (and its remaining
// norm when accepted), rn[src] its norm before orthogonalisation.
cudaError_t launch_gs_accept(long long n, int vt, void* R, int src, const double* scal, int n0,
                             int n1, double tol, const double* h1, const double* h2, double* Rt,
                             double* rn, int* ints, cudaStream_t s);
// Y[:, j] = sum_{i < kq} U[i + MAXB j] Q[:, i] for j < k <= kq (Y != Q)
cudaError_t launch_combine_multi(long long n, int vt, const void* Q, int kq, const double* U,
                                 int k, void* Y, cudaStream_t s);
// mixed-path CG (pairs x, r, p; float32 shadows p32 -> q32 and z32)
cudaError_t launch_dot_d2f(long long n, const void* a, const float* b, double* partials,
                           unsigned* counter, double* out, cudaStream_t s);
// x += alpha p, r -= alpha q, scal[rr] = |r|^2 with alpha = scal[num]/scal[den];
// with b non-null also b = float(r), zpre = omega dinv b (the next V-cycle's
// right-hand side and pre-smoothing from zero); host_rr (may be null): a
// device-accessible pointer to pinned host memory that also receives |r|^2
cudaError_t launch_cg_xr_d2(long long n, void* x, void* r, const void* p, const float* q,
                            double* scal, int num, int den, int rr, double* partials,
                            unsigned* counter, float* b, float* zpre, const float* dinv,
                            double omega, cudaStream_t s, double* host_rr = nullptr);
// p = z + beta p (num < 0: p = z), beta = scal[num]/scal[den]; p32 = float(p)
cudaError_t launch_cg_p_d2(long long n, void* p, float* p32, const float* z, const double* scal,
                           int num, int den, cudaStream_t s);
// small dense kernels on one thread block
cudaError_t launch_small_spd_inverse(int m, const int* m_dev, const double* A, double* Ainv,
                                     int* status, cudaStream_t s);
cudaError_t launch_small_matvec(int m, const int* m_dev, const double* A, const double* x,
                                double* y, double sign, cudaStream_t s);
cudaError_t launch_small_chol_solve(int m, const int* m_dev, const double* A, const double* b,
                                    double* x, int* status, cudaStream_t s);
// truncated SVD of the unit-column basis from its QR factor (one warp):
// U (ld MAXB) <- kept left singular vectors of Rt diag(rn)^-1 with
// sigma > tau sigma_1, ints[I_KRED] <- their count, sig <- singular values
cudaError_t launch_small_svd_trunc(int m, const int* kq_dev, const double* Rt, const double* rn,
                                   double tau, double* U, double* sig, int* ints,
                                   cudaStream_t s);
cudaError_t launch_eps(const double* scal, int rr, int f2, double* eps_dev, cudaStream_t s);

// ---- design-optimisation kernels (kernels_opt.cu) ----
cudaError_t launch_simp(long long nel, const double* rho, double E0, double Emin, double penal,
                        double* E64, float* E32, cudaStream_t s);
cudaError_t launch_delta(long long nel, const double* E, const double* Eprev, double* dE64,
                         float* dE32, float* Eprev32, cudaStream_t s);
cudaError_t launch_filter(int dim, const GridP& g, const StencilP& st, int mode,
                          const double* invHs, const double* in, double* out, cudaStream_t s);
cudaError_t launch_filter_norm(int dim, const GridP& g, const StencilP& st, double* invHs,
                               cudaStream_t s);
// 3D compliance and sensitivity in double-float arithmetic (mixed path);
// needs the Walsh blocks and an integer penal in [1, 9]
bool sensitivity_df_ok(int dim, double penal);
cudaError_t launch_sensitivity_df(const GridP& g, const uint8_t* mask, const double* wht,
                                  const double* u, const double* E, const double* rho,
                                  double penal, double E0, double Emin, double* dc,
                                  double* compliance, double* partials, unsigned* counter,
                                  cudaStream_t s);
// wht: host pointer to the float64 Walsh blocks of KE (3D), else null
// With v set (an adjoint field) the element term is v_e^T KE u_e instead of
// u_e^T KE u_e (generic kernel, no Walsh blocks) and `compliance` receives
// sum_e E_e v_e^T KE u_e.
cudaError_t launch_sensitivity(int dim, const GridP& g, const uint8_t* mask, const double* ke,
                               const double* wht, const double* u, const double* E,
                               const double* rho, double penal, double E0, double Emin,
                               double* dc, double* compliance, double* partials,
                               unsigned* counter, cudaStream_t s, const double* v = nullptr);
cudaError_t launch_oc_prep(long long nel, const double* rho, const double* dc,
                           const double* dv, double* a, double* scal, cudaStream_t s);
cudaError_t launch_oc_step(long long nel, const double* rho, const double* a,
                           const double* dv, double move, double target, double* scal,
                           double* partials, unsigned* counter, cudaStream_t s);
// bisection with stored move-limit bounds lo/hi (context path)
cudaError_t launch_oc_prep_b(long long nel, const double* rho, const double* dc,
                             const double* dv, double move, double* a, double* lo, double* hi,
                             double* scal, cudaStream_t s);
cudaError_t launch_oc_step_b(long long nel, const double* a, const double* lo, const double* hi,
                             const double* dv, double target, double* scal, double* partials,
                             unsigned* counter, cudaStream_t s);
// lambda search of the OC update: the candidate factors
// a = rho max(0, -dc/dv)^eta (float64 copy a64 for the final update; eta
// 1/2 for compliance) and the move limits and dv as double-float pairs; one
// launch narrows [l1, l2] eight-fold in double-float; rho_new =
// clamp(a lambda^-eta)
cudaError_t launch_oc_prep_d(long long nel, const double* rho, const double* dc,
                             const double* dv, double move, double* a64, void* a2, void* lo2,
                             void* hi2, void* dv2, double* scal, cudaStream_t s,
                             double eta = 0.5);
cudaError_t launch_oc_section(long long nel, const void* a2, const void* lo2, const void* hi2,
                              const void* dv2, double target, double* scal, double* partials,
                              unsigned* counter, cudaStream_t s, double eta = 0.5);
cudaError_t launch_oc_final(long long nel, double* rho, const double* a, double move,
                            double* scal, double* change_dev, double* partials,
                            unsigned* counter, cudaStream_t s, double eta = 0.5);
// Kc_E* += k w w^T for each spring: its fine DOF's interpolation weights w
// over the corners of one coarse element E* holding it (the Galerkin product
// P^T S P, element-wise; level 1 from the finest grid, stored matrices)
cudaError_t launch_spring_galerkin(int dim, int t, const GridP& gc, const GridP& gf,
                                   const Springs& sp, void* Kc, cudaStream_t s);

}  // namespace topo
