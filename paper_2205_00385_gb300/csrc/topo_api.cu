// C-ABI entry points of libtopo.so (declared in include/topo.h).
//
// The host side only sequences kernels on the context's stream and keeps
// bookkeeping (level geometry, PARM ring position, iteration counts); every
// arithmetic step of the solver path runs in the library's kernels.  Device
// memory comes exclusively from the caller's workspace.
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>

#include "kernels.h"

using namespace topo;

static std::string g_last_error;

namespace topo {

void note_launch(to_ctx* c) {
  if (c) c->launches++;
}

void set_global_error(const std::string& msg) { g_last_error = msg; }

}  // namespace topo

static to_status fail(to_ctx* c, to_status st, const std::string& msg) {
  if (c)
    c->last_error = msg;
  else
    g_last_error = msg;
  return st;
}

static to_status cuda_fail(to_ctx* c, const char* what, cudaError_t e) {
  return fail(c, TO_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define LAUNCH(c, expr, what)                                   \
  do {                                                          \
    cudaError_t _e = (expr);                                    \
    note_launch(c);                                             \
    if (_e != cudaSuccess) return cuda_fail((c), (what), _e);   \
  } while (0)

#define CUDA_TRY(c, expr, what)                                 \
  do {                                                          \
    cudaError_t _e = (expr);                                    \
    if (_e != cudaSuccess) return cuda_fail((c), (what), _e);   \
  } while (0)

// ---------------------------------------------------------------------------
// Profiling with CUDA events on the context stream
// ---------------------------------------------------------------------------
enum { PK_FINE32 = 0, PK_COARSE = 1, PK_VCYCLE = 2, PK_FINE_OTHER = 3, PK_N = 4 };

static cudaEvent_t ev_take(to_ctx* c) {
  cudaEvent_t e;
  if (!c->ev_pool.empty()) {
    e = c->ev_pool.back();
    c->ev_pool.pop_back();
    return e;
  }
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

struct ProfScope {
  to_ctx* c;
  int kind;
  double bytes;
  cudaEvent_t e0 = nullptr;
  ProfScope(to_ctx* c_, int k, double b = 0.0) : c(c_), kind(k), bytes(b) {
    if ((c->prof_mask >> kind) & 1u) {
      e0 = ev_take(c);
      if (e0) cudaEventRecord(e0, c->stream);
    }
  }
  ~ProfScope() {
    if (e0) {
      cudaEvent_t e1 = ev_take(c);
      if (e1) {
        cudaEventRecord(e1, c->stream);
        c->ev_used.push_back({kind, {e0, e1}});
        c->ev_bytes.push_back(bytes);
      }
    }
  }
};

// ---------------------------------------------------------------------------
// Element matrices and filter stencil (host tables, computed once per context)
// ---------------------------------------------------------------------------
// Unit-modulus element stiffness of a unit cell by 2-point Gauss quadrature,
// local node a = bx + 2by + 4bz, local DOF dim*a + c.
static void element_stiffness(int dim, double nu, double* KE) {
  const int npe = 1 << dim, nd = dim * npe;
  const double g = 0.5 / sqrt(3.0);
  const double gp[2] = {0.5 - g, 0.5 + g};
  const int ns = dim == 2 ? 3 : 6;
  double D[6][6] = {{0}};
  if (dim == 2) {
    const double s = 1.0 / (1.0 - nu * nu);
    D[0][0] = D[1][1] = s;
    D[0][1] = D[1][0] = s * nu;
    D[2][2] = s * (1.0 - nu) / 2.0;
  } else {
    const double lam = nu / ((1.0 + nu) * (1.0 - 2.0 * nu)), mu = 1.0 / (2.0 * (1.0 + nu));
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) D[i][j] = lam;
    for (int i = 0; i < 3; ++i) {
      D[i][i] = lam + 2.0 * mu;
      D[3 + i][3 + i] = mu;
    }
  }
  for (int q = 0; q < nd * nd; ++q) KE[q] = 0.0;
  const int nq = dim == 2 ? 4 : 8;
  for (int q = 0; q < nq; ++q) {
    double xi[3] = {gp[q & 1], gp[(q >> 1) & 1], gp[(q >> 2) & 1]};
    double w = dim == 2 ? 0.25 : 0.125;
    double B[6][24] = {{0}};
    for (int a = 0; a < npe; ++a) {
      double dN[3];
      for (int d = 0; d < dim; ++d) {
        double v = 1.0;
        for (int dd = 0; dd < dim; ++dd) {
          const int bit = (a >> dd) & 1;
          if (dd == d)
            v *= bit ? 1.0 : -1.0;
          else
            v *= bit ? xi[dd] : 1.0 - xi[dd];
        }
        dN[d] = v;
      }
      if (dim == 2) {
        B[0][2 * a] = dN[0];
        B[1][2 * a + 1] = dN[1];
        B[2][2 * a] = dN[1];
        B[2][2 * a + 1] = dN[0];
      } else {
        const int c = 3 * a;
        B[0][c] = dN[0];
        B[1][c + 1] = dN[1];
        B[2][c + 2] = dN[2];
        B[3][c] = dN[1];
        B[3][c + 1] = dN[0];
        B[4][c + 1] = dN[2];
        B[4][c + 2] = dN[1];
        B[5][c] = dN[2];
        B[5][c + 2] = dN[0];
      }
    }
    for (int i = 0; i < nd; ++i)
      for (int j = 0; j < nd; ++j) {
        double s = 0.0;
        for (int p = 0; p < ns; ++p)
          for (int r = 0; r < ns; ++r) s += B[p][i] * D[p][r] * B[r][j];
        KE[i * nd + j] += w * s;
      }
  }
}

// P_c: nodal values of child c's corners from its parent's corners
// (multilinear interpolation, per displacement component), nd x nd.
static void child_interp(int dim, int c, double* P) {
  const int npe = 1 << dim, nd = dim * npe;
  for (int a = 0; a < npe; ++a)
    for (int A = 0; A < npe; ++A) {
      double w = 1.0;
      for (int d = 0; d < dim; ++d) {
        const double pos = 0.5 * (((c >> d) & 1) + ((a >> d) & 1));
        w *= ((A >> d) & 1) ? pos : 1.0 - pos;
      }
      for (int ci = 0; ci < dim; ++ci)
        for (int cj = 0; cj < dim; ++cj) P[(dim * a + ci) * nd + dim * A + cj] = (ci == cj) ? w : 0.0;
    }
}

// out = P^T A P for nd x nd row-major matrices
static void triple(int nd, const double* P, const double* A, double* out) {
  std::vector<double> T(nd * nd);
  for (int i = 0; i < nd; ++i)
    for (int J = 0; J < nd; ++J) {
      double s = 0.0;
      for (int j = 0; j < nd; ++j) s += A[i * nd + j] * P[j * nd + J];
      T[i * nd + J] = s;
    }
  for (int I = 0; I < nd; ++I)
    for (int J = 0; J < nd; ++J) {
      double s = 0.0;
      for (int i = 0; i < nd; ++i) s += P[i * nd + I] * T[i * nd + J];
      out[I * nd + J] = s;
    }
}

// Q_c = P_c^T KE P_c for each child position c of a coarse element.
static void child_galerkin(int dim, const double* KE, double* Qc) {
  const int npe = 1 << dim, nd = dim * npe;
  std::vector<double> P(nd * nd);
  for (int c = 0; c < npe; ++c) {
    child_interp(dim, c, P.data());
    triple(nd, P.data(), KE, Qc + (size_t)c * nd * nd);
  }
}

// 3D: R_f = P_c1^T Q_c0 P_c1 for the 64 finest elements f = 8 c1 + c0 of a
// level-2 element (c1: level-1 parent inside it, c0: position in the parent).
static void grandchild_galerkin(const double* Qc, double* R) {
  std::vector<double> P(576);
  for (int c1 = 0; c1 < 8; ++c1) {
    child_interp(3, c1, P.data());
    for (int c0 = 0; c0 < 8; ++c0) triple(24, P.data(), Qc + (size_t)c0 * 576, R + (size_t)(8 * c1 + c0) * 576);
  }
}

static bool make_stencil(int dim, double rmin, StencilP* st) {
  const int R = (int)ceil(rmin);
  st->count = 0;
  for (int dz = (dim == 3 ? -R : 0); dz <= (dim == 3 ? R : 0); ++dz)
    for (int dy = -R; dy <= R; ++dy)
      for (int dx = -R; dx <= R; ++dx) {
        const double w = rmin - sqrt((double)(dx * dx + dy * dy + dz * dz));
        if (w <= 0.0) continue;
        if (st->count >= MAX_STENCIL) return false;
        st->d[st->count][0] = dx;
        st->d[st->count][1] = dy;
        st->d[st->count][2] = dz;
        st->w[st->count] = w;
        st->count++;
      }
  return true;
}

// ---------------------------------------------------------------------------
// Validation and workspace layout
// ---------------------------------------------------------------------------
static GridP level_grid(const to_mesh_desc& d, int l) {
  GridP g;
  g.nx = d.nel[0] >> l;
  g.ny = d.nel[1] >> l;
  g.nz = d.dim == 3 ? (d.nel[2] >> l) : 0;
  g.nnx = g.nx + 1;
  g.nny = g.ny + 1;
  g.nnz = d.dim == 3 ? g.nz + 1 : 1;
  g.nn = (long long)g.nnx * g.nny * g.nnz;
  g.nel = (long long)g.nx * g.ny * (d.dim == 3 ? g.nz : 1);
  return g;
}

static to_status validate(const to_mesh_desc* d, std::string* why) {
  if (!d) return *why = "desc is NULL", TO_E_INVALID;
  if (d->dim != 2 && d->dim != 3) return *why = "dim must be 2 or 3", TO_E_INVALID;
  if (d->mg_levels < 2 || d->mg_levels > MAXL)
    return *why = "mg_levels must be in [2, 10]", TO_E_INVALID;
  for (int i = 0; i < d->dim; ++i) {
    if (d->nel[i] < 1) return *why = "nel must be positive", TO_E_INVALID;
    const int f = 1 << (d->mg_levels - 1);
    if (d->nel[i] % f != 0)
      return *why = "every nel must be divisible by 2^(mg_levels-1)", TO_E_INVALID;
  }
  if (!(isfinite(d->E0) && isfinite(d->Emin) && d->Emin > 0.0 && d->E0 > d->Emin))
    return *why = "need 0 < Emin < E0", TO_E_INVALID;
  if (!(isfinite(d->nu) && d->nu > -1.0 && d->nu < 0.5)) return *why = "nu out of range", TO_E_INVALID;
  if (!(isfinite(d->penal) && d->penal >= 1.0)) return *why = "penal must be >= 1", TO_E_INVALID;
  if (!(isfinite(d->rmin) && d->rmin > 0.0 && d->rmin < 4.5))
    return *why = "rmin must be in (0, 4.5)", TO_E_INVALID;
  if (d->precision != TO_FP64 && d->precision != TO_MIXED)
    return *why = "precision must be TO_FP64 or TO_MIXED", TO_E_INVALID;
  if (d->n_parm < 1 || d->n_parm > MAXB || d->n_carm < 1 || d->n_carm > MAXB)
    return *why = "n_parm and n_carm must be in [1, 16]", TO_E_INVALID;
  GridP gc = level_grid(*d, d->mg_levels - 1);
  if (d->dim * gc.nn > 6144) return *why = "coarsest grid too large for the dense solve", TO_E_INVALID;
  return TO_OK;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Carver {
  char* base;
  size_t off = 0;
  template <class T>
  T* take(size_t count) {
    const size_t o = off;
    off = align256(off + count * sizeof(T));
    return base ? reinterpret_cast<T*>(base + o) : nullptr;
  }
};

static size_t carve(const to_mesh_desc& d, to_ctx* c, char* base) {
  Carver cv{base};
  const int dim = d.dim, npe = 1 << dim, nd = dim * npe, L = d.mg_levels;
  const bool mixed = d.precision == TO_MIXED;
  const size_t ts = mixed ? 4 : 8;
  GridP g0 = level_grid(d, 0);
  const long long nel = g0.nel, n = dim * g0.nn;
  const int Ns = d.n_parm, Nm = d.n_carm;
  double *E64 = cv.take<double>(nel), *Ep64 = cv.take<double>(nel), *dE64 = cv.take<double>(nel);
  double *rho = cv.take<double>(nel), *invHs = cv.take<double>(nel), *oca = cv.take<double>(nel);
  double *oclo = cv.take<double>(nel), *ochi = cv.take<double>(nel);
  double *oca2 = cv.take<double>(nel), *ocdv2 = cv.take<double>(nel);
  float *E32 = cv.take<float>(nel), *Ep32 = cv.take<float>(nel), *dE32 = cv.take<float>(nel);
  double* f = cv.take<double>(n);
  double* fd = cv.take<double>(n);
  double* w64 = (mixed && dim != 3) ? cv.take<double>(n) : nullptr;
  double *r = cv.take<double>(n), *z = cv.take<double>(n), *p = cv.take<double>(n),
         *q = cv.take<double>(n);
  float *p32 = cv.take<float>(n), *q32 = cv.take<float>(n);
  double *Phi = cv.take<double>((size_t)n * Ns), *KPhi = cv.take<double>((size_t)n * Ns);
  double *R = cv.take<double>((size_t)n * Nm), *Q = cv.take<double>((size_t)n * Nm);
  double* t = cv.take<double>(n);
  float* tc_bmat = dim == 3 ? cv.take<float>(2048) : nullptr;
  double* Qc64 = cv.take<double>((size_t)npe * nd * nd);
  float* Qc32 = cv.take<float>((size_t)npe * nd * nd);
  // 3D with >= 3 levels: level 1 is applied without stored matrices and
  // level 2 is formed from 64 grandchild tables
  const bool l1_implicit = dim == 3 && L >= 3;
  double* R2_64 = l1_implicit ? cv.take<double>((size_t)64 * 576) : nullptr;
  float* R2_32 = l1_implicit ? cv.take<float>((size_t)64 * 576) : nullptr;
  double* partials = cv.take<double>((size_t)RED_BLOCKS * MAXB * MAXB);
  unsigned* counters = cv.take<unsigned>(C_NCOUNTERS);
  double* scal = cv.take<double>(S_NSLOTS);
  double* small = cv.take<double>(SM_TOTAL);
  int* ints = cv.take<int>(I_NINTS);
  LevelBuf lv[MAXL];
  for (int l = 0; l < L; ++l) {
    GridP g = level_grid(d, l);
    const long long nl = dim * g.nn;
    lv[l].g = g;
    lv[l].n = nl;
    lv[l].mask = cv.take<uint8_t>(g.nn);
    lv[l].colfix = cv.take<uint8_t>((size_t)g.nnx * g.nny);
    lv[l].dinv = cv.take<char>(nl * ts);
    lv[l].b = cv.take<char>(nl * ts);
    lv[l].z = cv.take<char>(nl * ts);
    lv[l].z2 = cv.take<char>(nl * ts);
    lv[l].r = cv.take<char>(nl * ts);
    const bool stored = l >= 2 || (l == 1 && !l1_implicit);
    lv[l].Kc = stored ? (void*)cv.take<char>((size_t)tri_len(nd) * g.nel * ts) : nullptr;
    lv[l].S = stored ? (void*)cv.take<char>((size_t)stencil_values(dim, mixed ? T_F32 : T_F64, g) * ts)
                     : nullptr;
  }
  const long long nc = lv[L - 1].n;
  // the coarsest matrix and its inverse, sized for float64 (the storage of
  // the float64 path, and of the mixed path's coarse factorisation)
  void* Ad = cv.take<char>((size_t)nc * nc * 8);
  void* Ai = cv.take<char>((size_t)nc * nc * 8);
  if (c) {
    c->E64 = E64; c->Eprev64 = Ep64; c->dE64 = dE64; c->rho_phys = rho; c->invHs = invHs; c->oc_a = oca;
    c->oc_lo = oclo; c->oc_hi = ochi; c->oc_a2 = oca2; c->oc_dv2 = ocdv2;
    c->E32 = E32; c->Eprev32 = Ep32; c->dE32 = dE32; c->f = f; c->fd = fd; c->w64 = w64;
    c->r = r; c->z = z; c->p = p; c->q = q; c->p32 = p32; c->q32 = q32;
    c->Phi = Phi; c->KPhi = KPhi; c->R = R; c->Q = Q; c->t = t;
    c->Qc64 = Qc64; c->Qc32 = Qc32;
    c->tc_bmat = tc_bmat;
    c->l1_implicit = l1_implicit; c->R2_64 = R2_64; c->R2_32 = R2_32;
    c->partials = partials; c->counters = counters; c->scal = scal; c->small = small;
    c->ints = ints;
    for (int l = 0; l < L; ++l) c->lv[l] = lv[l];
    c->Adense = Ad; c->Ainv = Ai;
    c->nc = (int)nc;
  }
  return cv.off;
}

// ---------------------------------------------------------------------------
// Small device helpers used only at set-up
// ---------------------------------------------------------------------------
__global__ void k_node_mask(long long nn, int dim, const uint8_t* fixed, uint8_t* mask) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nn) return;
  unsigned m = 0;
  for (int c = 0; c < dim; ++c)
    if (fixed[dim * i + c]) m |= 1u << c;
  mask[i] = (uint8_t)m;
}

__global__ void k_coarse_mask(GridP gf, const uint8_t* mf, GridP gc, uint8_t* mc) {
  const long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= gc.nn) return;
  const int I = (int)(node % gc.nnx);
  const long long rest = node / gc.nnx;
  const int J = (int)(rest % gc.nny);
  const int K = (int)(rest / gc.nny);
  mc[node] = mf[2 * I + (long long)gf.nnx * (2 * J + (long long)gf.nny * 2 * K)];
}

// Flags a fixed fine DOF whose interpolation sources include a free coarse
// DOF (the Galerkin operators need fixed DOFs closed under interpolation),
// and loads on fixed DOFs.
__global__ void k_check_bc(GridP gf, const uint8_t* mf, GridP gc, const uint8_t* mc, int dim,
                           const double* f, int* flag) {
  const long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= gf.nn) return;
  const unsigned m = mf[node];
  if (!m) return;
  for (int c = 0; c < dim; ++c)
    if (((m >> c) & 1u) && f && f[dim * node + c] != 0.0) atomicOr(flag, 2);
  if (!mc) return;
  const int i = (int)(node % gf.nnx);
  const long long rest = node / gf.nnx;
  const int j = (int)(rest % gf.nny);
  const int k = (int)(rest / gf.nny);
  const int ni = (i & 1) ? 2 : 1, nj = (j & 1) ? 2 : 1, nk = (k & 1) ? 2 : 1;
  for (int a = 0; a < nk; ++a)
    for (int b = 0; b < nj; ++b)
      for (int cc = 0; cc < ni; ++cc) {
        const long long cn = ((i >> 1) + cc) + (long long)gc.nnx * (((j >> 1) + b) + (long long)gc.nny * ((k >> 1) + a));
        const unsigned mcv = mc[cn];
        for (int c = 0; c < dim; ++c)
          if (((m >> c) & 1u) && !((mcv >> c) & 1u)) atomicOr(flag, 1);
      }
}

// ---------------------------------------------------------------------------
// Public API
// ---------------------------------------------------------------------------
extern "C" {

to_status to_workspace_bytes(const to_mesh_desc* desc, int64_t* bytes) {
  std::string why;
  if (!bytes) return fail(nullptr, TO_E_INVALID, "bytes is NULL");
  to_status st = validate(desc, &why);
  if (st != TO_OK) return fail(nullptr, st, why);
  *bytes = (int64_t)carve(*desc, nullptr, nullptr) + 256;
  return TO_OK;
}

const char* to_last_error(const to_ctx* ctx) {
  return ctx ? ctx->last_error.c_str() : g_last_error.c_str();
}

static int mg_t(const to_ctx* c) { return c->mixed ? T_F32 : T_F64; }

to_status to_mesh_init(const to_mesh_desc* desc, const uint8_t* fixed_mask, const double* f,
                       void* workspace, int64_t ws_bytes, void* stream, to_ctx** out) {
  std::string why;
  if (!out) return fail(nullptr, TO_E_INVALID, "out is NULL");
  *out = nullptr;
  to_status st = validate(desc, &why);
  if (st != TO_OK) return fail(nullptr, st, why);
  if (!fixed_mask || !f || !workspace) return fail(nullptr, TO_E_INVALID, "NULL pointer argument");
  if (((uintptr_t)workspace) & 255) return fail(nullptr, TO_E_INVALID, "workspace not 256-byte aligned");
  const size_t need = carve(*desc, nullptr, nullptr);
  if (ws_bytes < (int64_t)need) return fail(nullptr, TO_E_OOM, "workspace too small");
  (void)cudaGetLastError();   // an error left by other code is not this call's
  to_ctx* c = new to_ctx();
  c->desc = *desc;
  c->dim = desc->dim;
  c->npe = 1 << c->dim;
  c->nd = c->dim * c->npe;
  c->L = desc->mg_levels;
  c->mixed = desc->precision == TO_MIXED;
  c->stream = (cudaStream_t)stream;
  carve(*desc, c, (char*)workspace);
  c->nel = c->lv[0].g.nel;
  c->nn = c->lv[0].g.nn;
  c->n = c->lv[0].n;
  c->parm_count = c->parm_head = c->carm_built = c->carm_qr = 0;
  c->have_density = false;
  c->hier_stale = true;
  c->launches = 0;
  c->prof_mask = 0u;
  c->n_vgraph = 0;
  c->vcycle_bytes = 0.0;
  c->coarse_t = c->mixed ? T_F32 : T_F64;
  c->coarse_shift = 0.0;
  for (int q = 0; q < 8; ++q) c->tuned_zc[q] = c->tuned_var[q] = 0;
  c->carm_flags = 0;
  c->use_tc = false;
  c->fuse_coarse = false;
  c->tall_tiles = false;
  c->work_list = false;
  c->vf_l0 = 0;
  c->springs = Springs();
  c->oc_eta = 0.5;
  c->host_rr = nullptr;
  c->host_rr_dev = nullptr;
  c->rr_event = nullptr;
  c->cap_stream = nullptr;
  if (!make_stencil(c->dim, desc->rmin, &c->stencil)) {
    delete c;
    return fail(nullptr, TO_E_INVALID, "filter stencil too large");
  }
  element_stiffness(c->dim, desc->nu, c->KE64);
  for (int q = 0; q < c->nd * c->nd; ++q) c->KE32[q] = (float)c->KE64[q];
  if (c->dim == 3) {
    wht_blocks(c->KE64, c->wht64);
    if (!df_blocks_ok(c->wht64)) {
      delete c;
      return fail(nullptr, TO_E_INVALID, "element Walsh blocks lack their structural zeros");
    }
    wht_blocks_pin_zeros(c->wht64, c->wht32);
  }
  c->df_ok = c->dim == 3;
  std::vector<double> Qc((size_t)c->npe * c->nd * c->nd);
  child_galerkin(c->dim, c->KE64, Qc.data());
  std::vector<float> Qc32(Qc.size());
  for (size_t q = 0; q < Qc.size(); ++q) Qc32[q] = (float)Qc[q];
  cudaStream_t s = c->stream;
  auto bad = [&](to_status code, const std::string& m) {
    g_last_error = m;
    delete c;
    return code;
  };
#define INIT_TRY(expr, what)                                              \
  do {                                                                    \
    cudaError_t _e = (expr);                                              \
    if (_e != cudaSuccess) return bad(TO_E_CUDA, std::string(what) + ": " + cudaGetErrorString(_e)); \
  } while (0)
  INIT_TRY(cudaMemcpyAsync(c->Qc64, Qc.data(), Qc.size() * 8, cudaMemcpyHostToDevice, s), "copy Qc");
  INIT_TRY(cudaMemcpyAsync(c->Qc32, Qc32.data(), Qc32.size() * 4, cudaMemcpyHostToDevice, s), "copy Qc32");
  std::vector<float> bpack(2048);
  if (c->dim == 3) {
    tc_pack_b(c->KE64, bpack.data());
    INIT_TRY(cudaMemcpyAsync(c->tc_bmat, bpack.data(), 2048 * 4, cudaMemcpyHostToDevice, s),
             "copy tensor-core B");
    INIT_TRY(cudaStreamSynchronize(s), "sync");
    INIT_TRY(tc_prepare(), "tensor-core operator set-up");
  }
  if (c->l1_implicit) {
    std::vector<double> R2((size_t)64 * 576);
    grandchild_galerkin(Qc.data(), R2.data());
    std::vector<float> R2f(R2.size());
    for (size_t q = 0; q < R2.size(); ++q) R2f[q] = (float)R2[q];
    INIT_TRY(cudaMemcpyAsync(c->R2_64, R2.data(), R2.size() * 8, cudaMemcpyHostToDevice, s), "copy R2");
    INIT_TRY(cudaMemcpyAsync(c->R2_32, R2f.data(), R2f.size() * 4, cudaMemcpyHostToDevice, s), "copy R2");
    INIT_TRY(cudaStreamSynchronize(s), "sync");
    for (int ch = 0; ch < 8; ++ch)
      for (int a = 0; a < 8; ++a)
        for (int cc = 0; cc < 3; ++cc)
          c->qdiag[(ch * 8 + a) * 3 + cc] = Qc[(size_t)ch * 576 + (3 * a + cc) * 24 + 3 * a + cc];
  }
  INIT_TRY(cudaMemcpyAsync(c->f, f, c->n * 8, cudaMemcpyDeviceToDevice, s), "copy f");
  if (c->mixed) INIT_TRY(launch_vconvert(c->n, V_F64, c->f, V_DF2, c->fd, s), "split f");
  INIT_TRY(cudaMemsetAsync(c->counters, 0, C_NCOUNTERS * sizeof(unsigned), s), "memset");
  INIT_TRY(cudaMemsetAsync(c->scal, 0, S_NSLOTS * 8, s), "memset");
  INIT_TRY(cudaMemsetAsync(c->ints, 0, I_NINTS * sizeof(int), s), "memset");
  INIT_TRY(cudaMemsetAsync(c->small, 0, SM_TOTAL * 8, s), "memset");
  k_node_mask<<<nblocks(c->nn, 256), 256, 0, s>>>(c->nn, c->dim, fixed_mask, c->lv[0].mask);
  INIT_TRY(cudaGetLastError(), "node mask");
  for (int l = 1; l < c->L; ++l) {
    k_coarse_mask<<<nblocks(c->lv[l].g.nn, 256), 256, 0, s>>>(c->lv[l - 1].g, c->lv[l - 1].mask,
                                                             c->lv[l].g, c->lv[l].mask);
    INIT_TRY(cudaGetLastError(), "coarse mask");
  }
  if (c->dim == 3) {
    pair_prepare();
    col_prepare();
    df_prepare();
  }
  // first level of the optional fused coarse stretch (TO_OPERATOR_FUSED_COARSE):
  // the first stored level whose stencil is small (a few MB)
  if (c->L >= 2 && vcycle_coarse_cluster(c->dim, mg_t(c), c->coarse_t) > 0) {
    const int first = c->l1_implicit ? 2 : 1;
    for (int l = first; l < c->L && l < VF_MAXL; ++l) {
      const double sbytes = (double)stencil_values(c->dim, mg_t(c), c->lv[l].g) *
                            (mg_t(c) == T_F64 ? 8.0 : 4.0);
      if (l == c->L - 1 || sbytes <= VF_MAX_STENCIL_BYTES) {
        c->vf_l0 = l;
        break;
      }
    }
    if (c->L > VF_MAXL) c->vf_l0 = 0;
  }
  (void)cudaGetLastError();
  for (int l = 0; l < c->L; ++l)
    INIT_TRY(launch_colfix(c->lv[l].g, c->lv[l].mask, c->lv[l].colfix, s), "column flags");
  for (int l = 0; l + 1 < c->L; ++l) {
    k_check_bc<<<nblocks(c->lv[l].g.nn, 256), 256, 0, s>>>(c->lv[l].g, c->lv[l].mask,
                                                          c->lv[l + 1].g, c->lv[l + 1].mask,
                                                          c->dim, l == 0 ? c->f : nullptr,
                                                          c->ints + I_STATUS);
    INIT_TRY(cudaGetLastError(), "bc check");
  }
  INIT_TRY(launch_filter_norm(c->dim, c->lv[0].g, c->stencil, c->invHs, s), "filter norm");
  INIT_TRY(launch_dot(c->n, c->f, c->f, c->partials, c->counters + C_DOT, c->scal + S_FNORM2, s),
           "norm f");
  double f2 = 0.0;
  int flag = 0;
  INIT_TRY(cudaMemcpyAsync(&f2, c->scal + S_FNORM2, 8, cudaMemcpyDeviceToHost, s), "read");
  INIT_TRY(cudaMemcpyAsync(&flag, c->ints + I_STATUS, 4, cudaMemcpyDeviceToHost, s), "read");
  INIT_TRY(cudaStreamSynchronize(s), "sync");
#undef INIT_TRY
  if (flag & 1) return bad(TO_E_INVALID, "supports not closed under coarse-grid interpolation");
  if (flag & 2) return bad(TO_E_INVALID, "load vector is nonzero on a fixed DOF");
  if (!(f2 > 0.0) || !isfinite(f2)) return bad(TO_E_INVALID, "load vector is zero or not finite");
  c->fnorm = sqrt(f2);
  cudaMemsetAsync(c->ints, 0, I_NINTS * sizeof(int), s);
  *out = c;
  return TO_OK;
}

void to_destroy(to_ctx* ctx) {
  if (!ctx) return;
  for (auto& u : ctx->ev_used) {
    cudaEventDestroy(u.second.first);
    cudaEventDestroy(u.second.second);
  }
  for (auto e : ctx->ev_pool) cudaEventDestroy(e);
  for (int q = 0; q < ctx->n_vgraph; ++q) cudaGraphExecDestroy(ctx->vgraph[q].exec);
  batch_forget(ctx);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  if (ctx->rr_event) cudaEventDestroy(ctx->rr_event);
  if (ctx->host_rr) cudaFreeHost(ctx->host_rr);
  delete ctx;
}

to_status to_set_density(to_ctx* c, const double* rho_phys) {
  if (!c || !rho_phys) return fail(c, TO_E_INVALID, "NULL argument");
  cudaStream_t s = c->stream;
  const to_mesh_desc& d = c->desc;
  CUDA_TRY(c, cudaMemcpyAsync(c->rho_phys, rho_phys, c->nel * 8, cudaMemcpyDeviceToDevice, s),
           "copy rho");
  if (c->have_density) std::swap(c->E64, c->Eprev64);
  LAUNCH(c, launch_simp(c->nel, c->rho_phys, d.E0, d.Emin, d.penal, c->E64, c->E32, s), "simp");
  if (!c->have_density)
    CUDA_TRY(c, cudaMemcpyAsync(c->Eprev64, c->E64, c->nel * 8, cudaMemcpyDeviceToDevice, s),
             "copy E");
  LAUNCH(c, launch_delta(c->nel, c->E64, c->Eprev64, c->dE64, c->dE32, c->Eprev32, s), "delta");
  c->have_density = true;
  c->hier_stale = true;
  return TO_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Internal solver pieces
// ---------------------------------------------------------------------------

static const void* coef_for(const to_ctx* c, int op, int tc) {
  if (tc == T_F64 || tc == T_DF) return op == TO_OP_K ? (const void*)c->E64
                        : op == TO_OP_KREF ? (const void*)c->Eprev64 : (const void*)c->dE64;
  return op == TO_OP_K ? (const void*)c->E32
         : op == TO_OP_KREF ? (const void*)c->Eprev32 : (const void*)c->dE32;
}

// autotuned kernel kind of a finest-grid launch (-1: not tuned)
static int tune_kind_fine(const to_ctx* c, int tc, int epi) {
  if (c->dim != 3) return -1;
  if (c->mixed ? tc == T_F32 : tc == T_F64)
    return epi == EPI_APPLY ? TO_TUNE_OP_APPLY : epi == EPI_RESID ? TO_TUNE_OP_RESID
                                                                  : TO_TUNE_OP_SMOOTH;
  if (tc == T_DF) return epi == EPI_RESID ? TO_TUNE_ACC_RESID : TO_TUNE_ACC_APPLY;
  return -1;
}

static ApplyArgs fine_args(const to_ctx* c, int op, int tc, int tx, int ty, const void* x,
                           void* y, const void* b, const void* dinv, int epi) {
  ApplyArgs a;
  a.dim = c->dim;
  a.g = c->lv[0].g;
  a.mask = c->lv[0].mask;
  a.tc = tc;
  a.tx = tx;
  a.ty = ty;
  a.expl = false;
  a.coef = coef_for(c, op, tc);
  a.Kc = nullptr;
  const bool wide = tc == T_F64 || tc == T_DF;
  a.ke = wide ? (const void*)c->KE64 : (const void*)c->KE32;
  a.wht = c->dim == 3 ? (wide ? (const void*)c->wht64 : (const void*)c->wht32) : nullptr;
  a.gal1 = false;
  a.gf = c->lv[0].g;
  a.S = nullptr;
  a.colfix = c->lv[0].colfix;
  a.x = x;
  a.y = y;
  a.b = b;
  a.dinv = dinv;
  a.omega = 0.6;
  a.dfix = op == TO_OP_DK ? 0.0 : 1.0;
  a.epi = epi;
  const int k = tune_kind_fine(c, tc, epi);
  a.zsplit = k >= 0 ? c->tuned_zc[k] : 0;
  a.variant = (k >= 0 ? c->tuned_var[k] : 0) | (c->tall_tiles ? 1 : 0) | (c->work_list ? 2 : 0);
  a.wl = c->counters + C_PAIR + 2 * (epi == EPI_APPLY ? 0 : epi == EPI_RESID ? 1 : 2);
  a.use_tc = c->use_tc;
  a.bmat = c->tc_bmat;
  a.status = c->ints + I_TIMEOUT;
  // the springs do not depend on the design: they cancel in dK
  if (op != TO_OP_DK) a.springs = c->springs;
  return a;
}

static ApplyArgs coarse_args(const to_ctx* c, int l, const void* x, void* y, const void* b,
                             int epi) {
  ApplyArgs a;
  const int t = mg_t(c);
  a.dim = c->dim;
  a.g = c->lv[l].g;
  a.mask = c->lv[l].mask;
  a.tc = t;
  a.tx = t;
  a.ty = t;
  a.expl = true;
  a.coef = nullptr;
  a.Kc = c->lv[l].Kc;
  a.ke = nullptr;
  a.wht = nullptr;
  a.gal1 = false;
  a.gf = c->lv[0].g;
  a.S = c->lv[l].S;
  a.colfix = c->lv[l].colfix;
  if (l == 1 && c->l1_implicit) {
    // level-1 Galerkin operator evaluated from the finest moduli
    a.expl = false;
    a.gal1 = true;
    a.coef = t == T_F64 ? (const void*)c->E64 : (const void*)c->E32;
    a.Kc = nullptr;
    a.wht = t == T_F64 ? (const void*)c->wht64 : (const void*)c->wht32;
    a.zsplit = epi == EPI_RESID ? c->tuned_zc[TO_TUNE_GAL1_RESID]
             : epi == EPI_SMOOTH ? c->tuned_zc[TO_TUNE_GAL1_SMOOTH] : 0;
  }
  a.x = x;
  a.y = y;
  a.b = b;
  a.dinv = c->lv[l].dinv;
  a.omega = 0.6;
  a.dfix = 1.0;
  a.epi = epi;
  return a;
}

// Algorithmic DRAM bytes of one operator launch: every input and output
// array touched once (the 3^dim neighbourhood reuse is not counted): x and
// y, the moduli (or the assembled stencil of a stored level), and the
// right-hand side and inverse diagonal of the fused epilogues.  The
// one-byte-per-node support masks are boundary data, not counted.
static double apply_bytes(const ApplyArgs& a) {
  const double sx = a.tx == T_F32 ? 4.0 : 8.0, sy = a.ty == T_F32 ? 4.0 : 8.0;
  const double sc = a.tc == T_F32 ? 4.0 : 8.0;
  const double n = (double)a.dim * (double)a.g.nn, nel = (double)a.g.nel;
  double b = n * (sx + sy);                             // x, y
  b += a.expl ? n * (a.dim == 3 ? 27 : 9) * a.dim * sc   // assembled stencil,
              : (a.gal1 ? 8.0 : 1.0) * nel * sc;         // or (child) moduli
  if (a.epi != EPI_APPLY) b += n * sx;                 // right-hand side
  if (a.epi == EPI_SMOOTH) b += n * sc;                // inverse diagonal
  return b;
}

static to_status run_op(to_ctx* c, const ApplyArgs& a, const char* what) {
  const bool fine32 = a.tc == T_F32 && a.tx == T_F32 && a.ty == T_F32;
  ProfScope ps(c, (a.expl || a.gal1) ? PK_COARSE : fine32 ? PK_FINE32 : PK_FINE_OTHER,
               apply_bytes(a));
  LAUNCH(c, launch_apply(a, c->stream), what);
  return TO_OK;
}

static to_status build_hierarchy(to_ctx* c) {
  // the launchers report cudaGetLastError(): clear what other code in this
  // thread may have left, so that it is not reported as this launch's error
  (void)cudaGetLastError();
  if (!c->have_density) return fail(c, TO_E_STATE, "to_set_density has not been called");
  cudaStream_t s = c->stream;
  const int t = mg_t(c);
  const void* E = t == T_F64 ? (const void*)c->E64 : (const void*)c->E32;
  const void* KE = t == T_F64 ? (const void*)c->KE64 : (const void*)c->KE32;
  const void* Qc = t == T_F64 ? (const void*)c->Qc64 : (const void*)c->Qc32;
  LAUNCH(c, launch_diag(c->dim, c->lv[0].g, c->lv[0].mask, t, false, E, nullptr, KE,
                        c->lv[0].dinv, s, c->springs), "diag 0");
  if (c->l1_implicit) {
    // level 1 stays implicit; level 2 straight from the finest moduli
    const void* R2 = t == T_F64 ? (const void*)c->R2_64 : (const void*)c->R2_32;
    LAUNCH(c, launch_diag_l1(t, c->lv[1].g, c->lv[0].g, c->lv[1].mask, c->qdiag, E,
                             c->lv[1].dinv, s), "diag 1");
    LAUNCH(c, launch_galerkin_l2(t, c->lv[2].g, c->lv[0].g, E, R2, c->lv[2].Kc, s), "galerkin 2");
  } else {
    LAUNCH(c, launch_galerkin_fine(c->dim, t, c->lv[1].g, c->lv[0].g, E, Qc, c->lv[1].Kc, s),
           "galerkin 1");
    LAUNCH(c, launch_spring_galerkin(c->dim, t, c->lv[1].g, c->lv[0].g, c->springs, c->lv[1].Kc,
                                     s), "springs 1");
  }
  const int lfirst = c->l1_implicit ? 3 : 2;
  for (int l = lfirst; l < c->L; ++l)
    LAUNCH(c, launch_galerkin_coarse(c->dim, t, c->lv[l].g, c->lv[l - 1].g, c->lv[l - 1].Kc,
                                     c->lv[l].Kc, s), "galerkin l");
  for (int l = c->l1_implicit ? 2 : 1; l < c->L; ++l) {
    LAUNCH(c, launch_diag(c->dim, c->lv[l].g, c->lv[l].mask, t, true, nullptr, c->lv[l].Kc,
                          nullptr, c->lv[l].dinv, s), "diag l");
    LAUNCH(c, launch_stencil_assemble(c->dim, t, c->lv[l].g, c->lv[l].mask, c->lv[l].Kc,
                                      c->lv[l].S, s), "stencil l");
  }
  const int Lc = c->L - 1;
  LAUNCH(c, launch_dense_assemble(c->dim, t, c->coarse_t, c->lv[Lc].g, c->lv[Lc].mask,
                                  c->lv[Lc].Kc, c->Adense, c->coarse_shift, s), "dense assemble");
  if (c->coarse_t == T_F32) {
    // float32 factorisation, checked: on high-contrast designs (near-void
    // regions at Emin / E0 = 1e-9) the float32 coarsest matrix can lose
    // positive definiteness; the context then factors it in float64 from
    // here on (the V-cycles captured with the float32 product are dropped)
    LAUNCH(c, launch_cholesky_inverse(T_F32, c->nc, c->Adense, c->Ainv, c->ints + I_COARSE, s),
           "coarse factor");
    int bad = 0;
    CUDA_TRY(c, cudaMemcpyAsync(&bad, c->ints + I_COARSE, sizeof(int), cudaMemcpyDeviceToHost, s),
             "read coarse status");
    CUDA_TRY(c, cudaStreamSynchronize(s), "sync");
    if (bad) {
      CUDA_TRY(c, cudaMemsetAsync(c->ints + I_COARSE, 0, sizeof(int), s), "reset");
      c->coarse_t = T_F64;
      for (int q = 0; q < c->n_vgraph; ++q) cudaGraphExecDestroy(c->vgraph[q].exec);
      c->n_vgraph = 0;
      LAUNCH(c, launch_dense_assemble(c->dim, t, c->coarse_t, c->lv[Lc].g, c->lv[Lc].mask,
                                      c->lv[Lc].Kc, c->Adense, c->coarse_shift, s),
             "dense assemble");
    }
  }
  if (c->coarse_t != T_F32)
    LAUNCH(c, launch_cholesky_inverse(c->coarse_t, c->nc, c->Adense, c->Ainv, c->ints + I_STATUS,
                                      s), "coarse factor");
  c->hier_stale = false;
  return TO_OK;
}

// zout (type zt: float64, or float32 in the mixed path) = V-cycle applied to
// r (storage rin_t: float64, or double-float pairs in the mixed path).  With
// pre set, the finest level's right-hand side b = r and pre-smoothing
// z = omega D^-1 b are already in place (written by the CG update).
// Algorithmic DRAM bytes of the V-cycle's kernels, each array a kernel
// touches counted once: presmoothing from zero reads the right-hand side and
// D^-1 and writes b and z; restriction reads the fine residual and writes
// the coarse right-hand side (and, pre-smoothing, reads D^-1 and writes z);
// interpolation reads the coarse correction and updates the fine iterate;
// the coarsest solve reads the dense inverse and two vectors.
static double vbytes_presmooth(long long n, int tin, int t) {
  return (double)n * ((tin == T_F64 || tin == T_D2 ? 8.0 : 4.0) + 3.0 * (t == T_F64 ? 8.0 : 4.0));
}
static double vbytes_restrict(long long nf, long long nc, int t, bool smooth) {
  const double ts = t == T_F64 ? 8.0 : 4.0;
  return ts * ((double)nf + (double)nc * (smooth ? 3.0 : 1.0));
}
static double vbytes_prolong(long long nf, long long nc, int t) {
  return (t == T_F64 ? 8.0 : 4.0) * (2.0 * (double)nf + (double)nc);
}
static double vbytes_coarse(long long nc, int ta, int t) {
  return (ta == T_F64 ? 8.0 : 4.0) * (double)nc * (double)nc +
         2.0 * (t == T_F64 ? 8.0 : 4.0) * (double)nc;
}

// clean: the right-hand side is zero on every fixed DOF (the solver's CG
// residual), so the finest level's vectors are too and its float32 operator
// needs to mask only the fixed rows' outputs.
static to_status vcycle(to_ctx* c, const void* rin, int rin_t, void* zout, int zt,
                        bool pre = false, bool clean = false) {
  cudaStream_t s = c->stream;
  const int t = mg_t(c);
  const int L = c->L;
  ProfScope ps(c, PK_VCYCLE);
  LevelBuf* lv = c->lv;
  double vb = 0.0;
  // finest level: smoothing from zero, residual, restriction
  if (!pre) {
    LAUNCH(c, launch_presmooth(t, rin_t, lv[0].n, rin, lv[0].b, lv[0].dinv, 0.6, lv[0].z, s),
           "presmooth 0");
    vb += vbytes_presmooth(lv[0].n, rin_t, t);
  }
  to_status st;
  {
    ApplyArgs a = fine_args(c, TO_OP_K, t, t, t, lv[0].z, lv[0].r, lv[0].b, lv[0].dinv,
                            EPI_RESID);
    a.clean_inputs = clean;
    vb += apply_bytes(a);
    if ((st = run_op(c, a, "resid 0")) != TO_OK) return st;
  }
  // restriction into level l also pre-smooths level l from a zero guess
  // (except on the coarsest level, which is solved exactly).  The residual of
  // a coarse level is zero on its fixed DOFs (its right-hand side and
  // zero-guess smoothing are), that of the finest level when the input is.
  auto restrict_into = [&](int l) {
    const bool smooth = l < L - 1;
    return launch_restrict(c->dim, t, lv[l - 1].g, lv[l - 1].mask, lv[l].g, lv[l].mask,
                           lv[l - 1].r, lv[l].b, smooth ? lv[l].dinv : nullptr, 0.6,
                           smooth ? lv[l].z : nullptr, clean || l >= 2, s);
  };
  // levels lf .. L-1 (lf = 0: none) run as one fused cluster launch
  const int lf = c->fuse_coarse ? c->vf_l0 : 0;
  if (lf != 1) {
    LAUNCH(c, restrict_into(1), "restrict 0");
    vb += vbytes_restrict(lv[0].n, lv[1].n, t, 1 < L - 1);
  }
  for (int l = 1; l < L - 1; ++l) {
    if (lf && l >= lf) break;
    ApplyArgs a = coarse_args(c, l, lv[l].z, lv[l].r, lv[l].b, EPI_RESID);
    a.clean_inputs = clean;
    vb += apply_bytes(a);
    if ((st = run_op(c, a, "resid l")) != TO_OK) return st;
    if (lf && l + 1 == lf) break;
    LAUNCH(c, restrict_into(l + 1), "restrict l");
    vb += vbytes_restrict(lv[l].n, lv[l + 1].n, t, l + 1 < L - 1);
  }
  if (lf) {
    VFuseArgs fa = {};
    fa.l0 = lf;
    fa.L = L;
    for (int l = lf - 1; l < L; ++l)
      fa.lv[l] = VFLevel{lv[l].g, lv[l].mask, lv[l].S, lv[l].dinv, lv[l].b, lv[l].z, lv[l].z2,
                         lv[l].r};
    fa.Ainv = c->Ainv;
    fa.nc = c->nc;
    fa.omega = 0.6;
    LAUNCH(c, launch_vcycle_coarse(c->dim, t, c->coarse_t, fa, s), "coarse levels (fused)");
    // the same algorithmic bytes as the separate launches
    vb += vbytes_restrict(lv[lf - 1].n, lv[lf].n, t, lf < L - 1);
    for (int l = lf; l < L - 1; ++l) {
      vb += apply_bytes(coarse_args(c, l, lv[l].z, lv[l].r, lv[l].b, EPI_RESID));
      vb += vbytes_restrict(lv[l].n, lv[l + 1].n, t, l + 1 < L - 1);
      vb += vbytes_prolong(lv[l].n, lv[l + 1].n, t);
      vb += apply_bytes(coarse_args(c, l, lv[l].z, lv[l].z2, lv[l].b, EPI_SMOOTH));
    }
    vb += vbytes_coarse(c->nc, c->coarse_t, t);
  } else {
    // coarsest grid: exact solve with the stored inverse
    LAUNCH(c, launch_dense_gemv(c->coarse_t, t, c->nc, c->Ainv, lv[L - 1].b, lv[L - 1].z2, s),
           "coarse solve");
    vb += vbytes_coarse(c->nc, c->coarse_t, t);
  }
  // upward: interpolate, post-smooth (result of level l lands in z2)
  for (int l = L - 2; l >= 1; --l) {
    if (lf && l >= lf) continue;
    LAUNCH(c, launch_prolong_add(c->dim, t, lv[l].g, lv[l].mask, lv[l + 1].g, lv[l + 1].z2,
                                 lv[l].z, s), "prolong l");
    vb += vbytes_prolong(lv[l].n, lv[l + 1].n, t);
    ApplyArgs a = coarse_args(c, l, lv[l].z, lv[l].z2, lv[l].b, EPI_SMOOTH);
    a.clean_inputs = clean;
    vb += apply_bytes(a);
    if ((st = run_op(c, a, "postsmooth l")) != TO_OK) return st;
  }
  LAUNCH(c, launch_prolong_add(c->dim, t, lv[0].g, lv[0].mask, lv[1].g, lv[1].z2, lv[0].z, s),
         "prolong 0");
  vb += vbytes_prolong(lv[0].n, lv[1].n, t);
  ApplyArgs a = fine_args(c, TO_OP_K, t, t, zt, lv[0].z, zout, lv[0].b, lv[0].dinv,
                          EPI_SMOOTH);
  a.clean_inputs = clean;
  vb += apply_bytes(a);
  ps.bytes = vb;
  c->vcycle_bytes = vb;
  return run_op(c, a, "postsmooth 0");
}

// The V-cycle's launch sequence depends only on buffer addresses fixed at
// set-up and on the coefficient array (which alternates between two buffers
// in float64), so it is captured once per (input, output, precision,
// coefficients) as a CUDA graph and replayed: one launch per preconditioner
// application instead of one per kernel, with no host gaps between kernels.
static to_status vcycle_graphed(to_ctx* c, const void* rin, int rin_t, void* zout, int zt,
                                bool pre = false) {
  const void* coef = mg_t(c) == T_F64 ? (const void*)c->E64 : (const void*)c->E32;
  to_ctx::VGraph* vg = nullptr;
  for (int q = 0; q < c->n_vgraph; ++q) {
    to_ctx::VGraph& v = c->vgraph[q];
    if (v.rin == rin && v.zout == zout && v.zt == zt && v.coef == coef && v.pre == pre) vg = &v;
  }
  if (!vg) {
    if (!c->cap_stream)
      CUDA_TRY(c, cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking),
               "capture stream");
    const cudaStream_t keep_stream = c->stream;
    const unsigned keep_prof = c->prof_mask;
    const long long keep_launches = c->launches;
    c->stream = c->cap_stream;
    c->prof_mask = 0u;
    cudaGraph_t graph = nullptr;
    to_status st = TO_OK;
    cudaError_t e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      st = vcycle(c, rin, rin_t, zout, zt, pre, true);
      const cudaError_t e2 = cudaStreamEndCapture(c->cap_stream, &graph);
      if (e == cudaSuccess) e = e2;
    }
    const long long captured = c->launches - keep_launches;
    c->stream = keep_stream;
    c->prof_mask = keep_prof;
    c->launches = keep_launches;
    cudaGraphExec_t exec = nullptr;
    if (st == TO_OK && e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (st != TO_OK) return st;
    if (e != cudaSuccess) return cuda_fail(c, "V-cycle graph", e);
    if (c->n_vgraph == 4) {
      cudaGraphExecDestroy(c->vgraph[0].exec);
      for (int q = 1; q < 4; ++q) c->vgraph[q - 1] = c->vgraph[q];
      c->n_vgraph = 3;
    }
    vg = &c->vgraph[c->n_vgraph++];
    *vg = to_ctx::VGraph{rin, zout, coef, zt, pre, exec, captured, c->vcycle_bytes};
  }
  ProfScope ps(c, PK_VCYCLE, vg->bytes);
  CUDA_TRY(c, cudaGraphLaunch(vg->exec, c->stream), "V-cycle graph launch");
  c->launches += vg->launches;
  return TO_OK;
}

static to_status read_scalar(to_ctx* c, const double* dev, double* host) {
  CUDA_TRY(c, cudaMemcpyAsync(host, dev, 8, cudaMemcpyDeviceToHost, c->stream), "read scalar");
  CUDA_TRY(c, cudaStreamSynchronize(c->stream), "sync");
  return TO_OK;
}

static to_status check_status(to_ctx* c) {
  int st[4] = {0, 0, 0, 0};
  CUDA_TRY(c, cudaMemcpyAsync(st, c->ints, sizeof(st), cudaMemcpyDeviceToHost, c->stream),
           "read status");
  CUDA_TRY(c, cudaStreamSynchronize(c->stream), "sync");
  if (st[I_TIMEOUT]) {
    cudaMemsetAsync(c->ints + I_TIMEOUT, 0, 4, c->stream);
    return fail(c, TO_E_TIMEOUT, "a bounded device wait expired (tensor-core operator)");
  }
  if (st[I_STATUS]) {
    cudaMemsetAsync(c->ints + I_STATUS, 0, 4, c->stream);
    return fail(c, TO_E_SINGULAR, "a factorisation met a non-positive pivot");
  }
  return TO_OK;
}

static int apply_tc(const to_ctx* c, int prec) {
  if (prec == TO_PREC_FP64) return T_F64;
  if (prec == TO_PREC_FP32) return T_F32;
  if (prec == TO_PREC_DF) return c->df_ok ? T_DF : T_F64;
  return c->mixed ? T_F32 : T_F64;
}

// Arithmetic of the float64-accurate products (true residuals, K R~): the
// FP64 path uses float64; the mixed path double-float where available.
static int accurate_tc(const to_ctx* c) { return (c->mixed && c->df_ok) ? T_DF : T_F64; }

static to_status apply_op(to_ctx* c, int op, int prec, const double* x, double* y) {
  const int tc = apply_tc(c, prec);
  const ApplyArgs a32 = fine_args(c, op, tc, T_F32, T_F32, c->p32, c->q32, nullptr, nullptr,
                                  EPI_APPLY);
  if (prec == TO_PREC_FP32 && pair_apply_ok(a32)) {
    // float32 storage end to end: the operator that runs inside the mixed solver
    LAUNCH(c, launch_convert(T_F64, T_F32, c->n, x, c->p32, c->stream), "convert x");
    to_status st = run_op(c, a32, "apply");
    if (st != TO_OK) return st;
    LAUNCH(c, launch_convert(T_F32, T_F64, c->n, c->q32, y, c->stream), "convert y");
    return TO_OK;
  }
  return run_op(c, fine_args(c, op, tc, T_F64, T_F64, x, y, nullptr, nullptr, EPI_APPLY),
                "apply");
}

// Storage of the long float64-accurate vectors (CG iterate, r, p; Phi,
// KPhi, R, Q, t): float64 on the FP64 path, double-float pairs on the mixed
// path (arithmetic on the FP32 pipe; GB300's FP64 pipe is 1/128 of FP32).
static int vt(const to_ctx* c) { return c->mixed ? V_DF2 : V_F64; }
static int vt_code(const to_ctx* c) { return c->mixed ? T_D2 : T_F64; }

// y = op(x) in the context's apply precision, x and y in vector storage:
// float64 on the FP64 path; float32 through the shadows p32 -> q32 (the
// solver's float32 operator) on the mixed path
static to_status apply_vec(to_ctx* c, int op, const double* x, double* y) {
  if (!c->mixed)
    return run_op(c, fine_args(c, op, T_F64, T_F64, T_F64, x, y, nullptr, nullptr, EPI_APPLY),
                  "apply");
  LAUNCH(c, launch_convert(T_D2, T_F32, c->n, x, c->p32, c->stream), "round x");
  to_status st = run_op(c, fine_args(c, op, T_F32, T_F32, T_F32, c->p32, c->q32, nullptr,
                                     nullptr, EPI_APPLY), "apply");
  if (st != TO_OK) return st;
  LAUNCH(c, launch_convert(T_F32, T_D2, c->n, c->q32, y, c->stream), "widen y");
  return TO_OK;
}

// float64-accurate y = op(x) (EPI_APPLY) or y = f - op(x) (EPI_RESID), x
// and y in vector storage: float64 operator, double-float operator on pairs,
// or (mixed 2D) the float64 operator through float64 scratch
static to_status apply_accurate_vec(to_ctx* c, int op, const double* x, double* y, int epi) {
  const bool resid = epi == EPI_RESID;
  if (!c->mixed)
    return run_op(c, fine_args(c, op, T_F64, T_F64, T_F64, x, y, resid ? c->f : nullptr, nullptr,
                               epi), "accurate apply");
  if (c->df_ok)
    return run_op(c, fine_args(c, op, T_DF, T_D2, T_D2, x, y, resid ? c->fd : nullptr, nullptr,
                               epi), "accurate apply");
  LAUNCH(c, launch_vconvert(c->n, V_DF2, x, V_F64, c->q, c->stream), "widen x");
  to_status st = run_op(c, fine_args(c, op, T_F64, T_F64, T_F64, c->q, c->w64,
                                     resid ? c->f : nullptr, nullptr, epi), "accurate apply");
  if (st != TO_OK) return st;
  LAUNCH(c, launch_vconvert(c->n, V_F64, c->w64, V_DF2, y, c->stream), "split y");
  return TO_OK;
}

static to_status parm_push(to_ctx* c, const double* u) {
  cudaStream_t s = c->stream;
  const int Ns = c->desc.n_parm;
  const int slot = c->parm_head;
  double* col = c->Phi + (size_t)slot * c->n;
  LAUNCH(c, launch_vconvert(c->n, V_F64, u, vt(c), col, s), "copy");
  LAUNCH(c, launch_vdot(c->n, vt(c), col, col, c->partials, c->counters + C_DOT, c->scal + S_NRM,
                        s), "norm");
  LAUNCH(c, launch_vscale_inv_sqrt(c->n, vt(c), col, c->scal + S_NRM, s), "scale");
  c->parm_head = (c->parm_head + 1) % Ns;
  c->parm_count = std::min(c->parm_count + 1, Ns);
  return TO_OK;
}

extern "C" {

to_status to_apply(to_ctx* c, int32_t op, int32_t prec, const double* x, double* y) {
  if (!c || !x || !y || x == y) return fail(c, TO_E_INVALID, "bad arguments");
  if (op < TO_OP_K || op > TO_OP_DK || prec < 0 || prec > 3) return fail(c, TO_E_INVALID, "bad op");
  if (!c->have_density) return fail(c, TO_E_STATE, "to_set_density has not been called");
  return apply_op(c, op, prec, x, y);
}

to_status to_vcycle(to_ctx* c, const double* r, double* z) {
  if (!c || !r || !z || r == z) return fail(c, TO_E_INVALID, "bad arguments");
  if (c->hier_stale) {
    to_status st = build_hierarchy(c);
    if (st != TO_OK) return st;
  }
  if (!c->mixed) return vcycle(c, r, T_F64, z, T_F64);
  to_status st = vcycle(c, r, T_F64, c->lv[0].z2, T_F32);
  if (st != TO_OK) return st;
  LAUNCH(c, launch_convert(T_F32, T_F64, c->n, c->lv[0].z2, z, c->stream), "convert");
  return TO_OK;
}

to_status to_level_info(to_ctx* c, int32_t level, int32_t nel_out[3], int64_t* ndof) {
  if (!c || level < 0 || level >= c->L || !nel_out || !ndof) return fail(c, TO_E_INVALID, "bad level");
  nel_out[0] = c->lv[level].g.nx;
  nel_out[1] = c->lv[level].g.ny;
  nel_out[2] = c->lv[level].g.nz;
  *ndof = c->lv[level].n;
  return TO_OK;
}

to_status to_level_apply(to_ctx* c, int32_t level, const double* x, double* y) {
  if (!c || !x || !y || level < 1 || level >= c->L) return fail(c, TO_E_INVALID, "bad arguments");
  if (c->hier_stale) {
    to_status st = build_hierarchy(c);
    if (st != TO_OK) return st;
  }
  cudaStream_t s = c->stream;
  LevelBuf& L = c->lv[level];
  const int t = mg_t(c);
  LAUNCH(c, launch_convert(T_F64, t, L.n, x, L.z2, s), "convert");
  LAUNCH(c, launch_apply(coarse_args(c, level, L.z2, L.r, nullptr, EPI_APPLY), s), "level apply");
  LAUNCH(c, launch_convert(t, T_F64, L.n, L.r, y, s), "convert");
  return TO_OK;
}

to_status to_mgcg_solve(to_ctx* c, double rtol, int32_t maxit, int32_t flags, double* u,
                        int32_t* iters, double* relres) {
  if (!c || !u) return fail(c, TO_E_INVALID, "NULL argument");
  if (!(rtol >= 0.0) || !isfinite(rtol) || maxit < 1) return fail(c, TO_E_INVALID, "bad rtol/maxit");
  if (!c->have_density) return fail(c, TO_E_STATE, "to_set_density has not been called");
  cudaStream_t s = c->stream;
  to_status st;
  if (c->hier_stale && (st = build_hierarchy(c)) != TO_OK) return st;
  if (!c->host_rr) {
    // 64 bytes of pinned host memory per context, mapped into the device's
    // address space: the CG update kernel writes |r|^2 there itself and the
    // host waits on an event recorded after it
    void* h = nullptr;
    CUDA_TRY(c, cudaHostAlloc(&h, 64, cudaHostAllocMapped), "pinned residual slot");
    c->host_rr = static_cast<double*>(h);
    void* d = nullptr;
    CUDA_TRY(c, cudaHostGetDevicePointer(&d, h, 0), "mapped residual slot");
    c->host_rr_dev = static_cast<double*>(d);
  }
  if (!c->rr_event)
    CUDA_TRY(c, cudaEventCreateWithFlags(&c->rr_event, cudaEventDisableTiming), "rr event");
  const long long n = c->n;
  // Mixed path: the iterate x, r and p are double-float pairs (x in the
  // otherwise unused float64 z buffer); the operator and the V-cycle work on
  // float32 shadows (p32 -> q32, z32); dot products are double-float.
  // FP64 path: everything float64, x = u.
  const bool mixed = c->mixed;
  double* x = mixed ? c->z : u;
  const bool warm = (flags & TO_SOLVE_WARM_START) != 0;
  if (mixed && warm) {
    LAUNCH(c, launch_vconvert(n, V_F64, u, V_DF2, x, s), "split u");
    // the solution is zero on the fixed DOFs; a warm start that is not gets
    // those entries cleared, so that every vector of the solve is (the
    // float32 operator relies on it)
    LAUNCH(c, launch_zero_fixed(c->nn, c->dim, c->lv[0].mask, V_DF2, x, s), "clear fixed");
  } else if (!warm) {
    CUDA_TRY(c, cudaMemsetAsync(x, 0, n * 8, s), "zero x");
  } else {
    LAUNCH(c, launch_zero_fixed(c->nn, c->dim, c->lv[0].mask, V_F64, x, s), "clear fixed");
  }
  // r = f - K x with the float64-accurate operator (the true residual)
  auto true_residual = [&](double* rr_out) -> to_status {
    to_status e;
    if ((e = apply_accurate_vec(c, TO_OP_K, x, c->r, EPI_RESID)) != TO_OK) return e;
    LAUNCH(c, launch_vdot(n, vt(c), c->r, c->r, c->partials, c->counters + C_DOT,
                          c->scal + S_RR, s), "rr");
    return read_scalar(c, c->scal + S_RR, rr_out);
  };
  double rr = 0.0;
  if ((st = true_residual(&rr)) != TO_OK) return st;
  double rel = sqrt(rr) / c->fnorm;
  double rr_max = rr;          // largest residual since the last true-residual update
  int it = 0;
  bool conv = rel < rtol;
  float* z32 = static_cast<float*>(c->lv[0].z2);
  // mixed path: the CG update also writes the next V-cycle's right-hand side
  // and pre-smoothing (lv[0].b, lv[0].z); a true residual invalidates them
  bool pre = false;
  auto precondition = [&](int slot) -> to_status {
    to_status e;
    if (mixed) {
      if ((e = vcycle_graphed(c, c->r, T_D2, z32, T_F32, pre)) != TO_OK) return e;
      LAUNCH(c, launch_dot_d2f(n, c->r, z32, c->partials, c->counters + C_DOT, c->scal + slot, s),
             "rz");
    } else {
      if ((e = vcycle_graphed(c, c->r, T_F64, c->z, T_F64)) != TO_OK) return e;
      LAUNCH(c, launch_dot(n, c->r, c->z, c->partials, c->counters + C_DOT, c->scal + slot, s),
             "rz");
    }
    return TO_OK;
  };
  if (!conv) {
    if ((st = precondition(S_RZ0)) != TO_OK) return st;
    if (mixed)
      LAUNCH(c, launch_cg_p_d2(n, c->p, c->p32, z32, c->scal, -1, 0, s), "p = z");
    else
      LAUNCH(c, launch_copy(n, c->z, c->p, s), "p = z");
    int cur = S_RZ0, nxt = S_RZ1;
    // Precision escalation (mixed path): q = K p in float32 carries ~1e-4
    // relative error on smooth search directions (K cancels by 1e3-1e4
    // there), and on some designs CG stagnates on it, the recursive and
    // true residuals stuck together.  Healthy convergence gains >= 10x in
    // 16 iterations; when the residual fails to halve over 16 iterations,
    // the rest of the solve forms q with the double-float operator (then
    // rounded to float32, which loses nothing to cancellation) and CG
    // restarts from the true residual.
    bool accurate_q = false;
    double rel_window = rel;
    int it_window = 0;
    for (it = 1; it <= maxit; ++it) {
      if (mixed && accurate_q) {
        if ((st = apply_accurate_vec(c, TO_OP_K, c->p, c->t, EPI_APPLY)) != TO_OK) return st;
        LAUNCH(c, launch_convert(T_D2, T_F32, n, c->t, c->q32, s), "q to float32");
      } else if (mixed) {
        ApplyArgs a = fine_args(c, TO_OP_K, T_F32, T_F32, T_F32, c->p32, c->q32, nullptr,
                                nullptr, EPI_APPLY);
        a.clean_inputs = true;   // p is zero on the fixed DOFs
        if ((st = run_op(c, a, "q = K p")) != TO_OK) return st;
      }
      if (mixed) {
        LAUNCH(c, launch_dot_d2f(n, c->p, c->q32, c->partials, c->counters + C_DOT,
                                 c->scal + S_PQ, s), "pq");
        LAUNCH(c, launch_cg_xr_d2(n, x, c->r, c->p, c->q32, c->scal, cur, S_PQ, S_RR,
                                  c->partials, c->counters + C_UPD,
                                  static_cast<float*>(c->lv[0].b), static_cast<float*>(c->lv[0].z),
                                  static_cast<const float*>(c->lv[0].dinv), 0.6, s,
                                  c->host_rr_dev),
               "x, r update");
        pre = true;
      } else {
        ApplyArgs a = fine_args(c, TO_OP_K, T_F64, T_F64, T_F64, c->p, c->q, nullptr, nullptr,
                                EPI_APPLY);
        a.clean_inputs = true;   // p is zero on the fixed DOFs
        if ((st = run_op(c, a, "q = K p")) != TO_OK) return st;
        LAUNCH(c, launch_dot(n, c->p, c->q, c->partials, c->counters + C_DOT, c->scal + S_PQ, s),
               "pq");
        LAUNCH(c, launch_cg_xr(n, x, c->r, c->p, c->q, c->scal, cur, S_PQ, S_RR, c->partials,
                               c->counters + C_UPD, s, c->host_rr_dev), "x, r update");
      }
      // |r|^2 goes to the host, and the next preconditioner application is
      // enqueued before the host waits for it: the V-cycle runs while the
      // host reads the residual and decides.  The preconditioner writes only
      // its own scratch and scal[nxt], so when the loop stops (or a true
      // residual replaces r) its result is discarded (or recomputed) and
      // the iterates are the same as with the read first.
      // (the update kernel writes it into the mapped host slot itself)
      CUDA_TRY(c, cudaEventRecord(c->rr_event, s), "rr event");
      bool fresh = it < maxit;
      if (fresh && (st = precondition(nxt)) != TO_OK) return st;
      CUDA_TRY(c, cudaEventSynchronize(c->rr_event), "wait rr");
      rr = *reinterpret_cast<volatile double*>(c->host_rr);
      rel = sqrt(rr) / c->fnorm;
      if (!isfinite(rel)) return fail(c, TO_E_SINGULAR, "CG breakdown (non-finite residual)");
      // Reliable updates: with a float32 operator the recursive residual
      // drifts from f - K x, so it is replaced by the float64-accurate true
      // residual whenever it has dropped 100x since the last replacement and
      // before convergence is declared.  The search direction is kept when
      // the two agree; when the true residual is more than 1.5x the
      // recursive one the recursion has drifted (its directions were built
      // for a different residual), and CG restarts from the true residual
      // (p = z).
      bool restart = false;
      bool escalate = false;
      if (mixed && !accurate_q && it - it_window >= 16) {
        escalate = rel > 0.5 * rel_window;
        rel_window = rel;
        it_window = it;
      }
      if (mixed && (rel < rtol || rr < 1e-4 * rr_max || escalate)) {
        const double rr_rec = rr;
        if ((st = true_residual(&rr)) != TO_OK) return st;
        pre = false;
        fresh = false;
        restart = escalate || rr > 2.25 * rr_rec;
        rel = sqrt(rr) / c->fnorm;
        rr_max = rr;
        if (escalate) accurate_q = true;
      }
      rr_max = std::max(rr_max, rr);
      if (rel < rtol) {
        conv = true;
        break;
      }
      if (it == maxit) break;
      if (!fresh && (st = precondition(nxt)) != TO_OK) return st;
      if (mixed)
        LAUNCH(c, launch_cg_p_d2(n, c->p, c->p32, z32, c->scal, restart ? -1 : nxt, cur, s),
               "p update");
      else
        LAUNCH(c, launch_cg_p(n, c->p, c->z, c->scal, nxt, cur, s), "p update");
      std::swap(cur, nxt);
    }
    if (it > maxit) it = maxit;
    // the iterate back to float64 (untouched when no step was taken)
    if (mixed) LAUNCH(c, launch_vconvert(n, V_DF2, x, V_F64, u, s), "widen x");
  }
  if (iters) *iters = it;
  if (relres) *relres = rel;
  if ((st = check_status(c)) != TO_OK) return st;
  if (flags & TO_SOLVE_PUSH_PARM) {
    if ((st = parm_push(c, u)) != TO_OK) return st;
  }
  if (!conv) return fail(c, TO_E_NOT_CONVERGED, "MGCG reached maxit");
  return TO_OK;
}

to_status to_parm_push(to_ctx* c, const double* u) {
  if (!c || !u) return fail(c, TO_E_INVALID, "NULL argument");
  return parm_push(c, u);
}

to_status to_parm_count(to_ctx* c, int32_t* count) {
  if (!c || !count) return fail(c, TO_E_INVALID, "NULL argument");
  *count = c->parm_count;
  return TO_OK;
}

to_status to_parm_reset(to_ctx* c) {
  if (!c) return fail(c, TO_E_INVALID, "NULL argument");
  c->parm_count = c->parm_head = 0;
  return TO_OK;
}

to_status to_carm_build(to_ctx* c, const double* u_last) {
  if (!c || !u_last) return fail(c, TO_E_INVALID, "NULL argument");
  if (!c->have_density) return fail(c, TO_E_STATE, "to_set_density has not been called");
  if (c->parm_count < c->desc.n_parm) return fail(c, TO_E_STATE, "PARM is not full");
  cudaStream_t s = c->stream;
  const long long n = c->n;
  const int Ns = c->desc.n_parm, m = c->desc.n_carm;
  to_status st;
  double* small = c->small;
  const int v = vt(c);
  c->carm_built = c->carm_qr = 0;
  // Both products below use the float64-accurate operator in either
  // precision: for smooth displacement fields K x cancels heavily, and a
  // float32 product would leave the basis with errors of ~1e-3.
  // K_Phi = Phi^T K_ref Phi  (Eq. 15)
  for (int i = 0; i < Ns; ++i)
    if ((st = apply_accurate_vec(c, TO_OP_KREF, c->Phi + (size_t)i * n, c->KPhi + (size_t)i * n,
                                 EPI_APPLY)) != TO_OK)
      return st;
  LAUNCH(c, launch_gram_sym(n, v, c->Phi, c->KPhi, Ns, small + SM_KPHI, Ns, c->partials,
                            c->counters + C_MULTI, s), "K_Phi");
  LAUNCH(c, launch_small_spd_inverse(Ns, nullptr, small + SM_KPHI, small + SM_KPHI_INV,
                                     c->ints + I_STATUS, s), "K_Phi inverse");
  // r_1 = u_last (or Phi K_Phi^{-1} Phi^T f, the alternative of Fig. 2);
  // r_i = -Phi K_Phi^{-1} Phi^T dK r_{i-1}  (Eq. 18-20, 26)
  if (c->carm_flags & TO_CARM_R1_PROJECTED_LOAD) {
    const double* fv = c->mixed ? c->fd : c->f;
    LAUNCH(c, launch_gram(n, v, c->Phi, Ns, nullptr, fv, 1, nullptr, small + SM_Z, Ns,
                          c->partials, c->counters + C_MULTI, s), "Phi^T f");
    LAUNCH(c, launch_small_matvec(Ns, nullptr, small + SM_KPHI_INV, small + SM_Z, small + SM_W,
                                  1.0, s), "K_Phi^-1 Phi^T f");
    LAUNCH(c, launch_combine(n, v, c->Phi, Ns, nullptr, small + SM_W, 1.0, 0.0, c->R, v, nullptr,
                             nullptr, c->partials, c->counters + C_UPD, s), "r1");
  } else {
    LAUNCH(c, launch_vconvert(n, V_F64, u_last, v, c->R, s), "r1");
  }
  for (int i = 1; i < m; ++i) {
    if ((st = apply_accurate_vec(c, TO_OP_DK, c->R + (size_t)(i - 1) * n, c->t, EPI_APPLY)) !=
        TO_OK)
      return st;
    LAUNCH(c, launch_gram(n, v, c->Phi, Ns, nullptr, c->t, 1, nullptr, small + SM_Z, Ns,
                          c->partials, c->counters + C_MULTI, s), "Phi^T t");
    LAUNCH(c, launch_small_matvec(Ns, nullptr, small + SM_KPHI_INV, small + SM_Z, small + SM_W,
                                  -1.0, s), "K_Phi^-1 z");
    LAUNCH(c, launch_combine(n, v, c->Phi, Ns, nullptr, small + SM_W, 1.0, 0.0,
                             c->R + (size_t)i * n, v, nullptr, nullptr, c->partials,
                             c->counters + C_UPD, s), "r_i");
  }
  // Eq. 21 (R = R~ Sigma V^T, truncated).  QR of R in place by classical
  // Gram-Schmidt run twice per column: Q lands in the first kq columns of R,
  // the triangular factor in small[SM_RT].  A column left with <= 1e-10 of
  // its norm after both passes is numerically dependent on the earlier ones
  // and gets no column of Q (its projections stay in the factor).
  CUDA_TRY(c, cudaMemsetAsync(c->ints + I_KCOUNT, 0, sizeof(int), s), "reset k");
  for (int i = 0; i < m; ++i) {
    double* ri = c->R + (size_t)i * n;
    const int bound = std::max(i, 1);   // accepted columns so far <= i
    LAUNCH(c, launch_vdot(n, v, ri, ri, c->partials, c->counters + C_DOT, c->scal + S_NRM0, s),
           "|r|");
    // two classical passes: projections, then the first update fused with
    // the second pass's projections, then the second update, which also
    // returns |r_i|^2 after them
    LAUNCH(c, launch_gram(n, v, c->R, bound, c->ints + I_KCOUNT, ri, 1, nullptr, small + SM_H,
                          MAXB, c->partials, c->counters + C_MULTI, s), "GS dots");
    LAUNCH(c, launch_combine_dots(n, v, c->R, bound, c->ints + I_KCOUNT, small + SM_H, ri,
                                  small + SM_H2, c->partials, c->counters + C_MULTI, s),
           "GS axpy + dots");
    LAUNCH(c, launch_combine(n, v, c->R, bound, c->ints + I_KCOUNT, small + SM_H2, -1.0, 1.0, ri,
                             v, nullptr, c->scal + S_NRM1, c->partials, c->counters + C_UPD, s),
           "GS axpy");
    LAUNCH(c, launch_gs_accept(n, v, c->R, i, c->scal, S_NRM0, S_NRM1, TO_QR_DEPENDENT_TOL,
                               small + SM_H, small + SM_H2, small + SM_RT, small + SM_RN, c->ints,
                               s), "GS accept");
  }
  // singular values of the unit-column basis from the small factor; the
  // directions with sigma > TO_CARM_SVD_TOL sigma_1 span R~
  LAUNCH(c, launch_small_svd_trunc(m, c->ints + I_KCOUNT, small + SM_RT, small + SM_RN,
                                   TO_CARM_SVD_TOL, small + SM_U, small + SM_SIG, c->ints, s),
         "truncated SVD");
  int kk[3] = {0, 0, 0};
  CUDA_TRY(c, cudaMemcpyAsync(kk, c->ints, sizeof(kk), cudaMemcpyDeviceToHost, s), "read counts");
  CUDA_TRY(c, cudaStreamSynchronize(s), "sync");
  const int kq = kk[I_KCOUNT], k = kk[I_KRED];
  if (kq < 1 || k < 1) return fail(c, TO_E_SINGULAR, "CARM basis is empty");
  // R~ = Q U into the Q buffer, then the two buffers trade places (both hold
  // n x N_m values of the same storage)
  LAUNCH(c, launch_combine_multi(n, v, c->R, kq, small + SM_U, k, c->Q, s), "R~ = Q U");
  std::swap(c->R, c->Q);
  c->carm_qr = kq;
  c->carm_built = k;
  return TO_OK;
}

// process-wide cache of tuned chunk lengths: (device, kernel, grid) -> layers
static std::mutex g_tune_mu;
static std::map<std::tuple<int, int, long long, long long, long long>, std::pair<int, int>>
    g_tune_cache;   // -> (layers per chunk, register variant)

to_status to_autotune(to_ctx* c, int32_t reps, to_tune_result* results, int32_t cap,
                      int32_t* count) {
  if (!c || !count || reps < 1 || cap < 0 || (cap > 0 && !results))
    return fail(c, TO_E_INVALID, "bad arguments");
  if (!c->have_density) return fail(c, TO_E_STATE, "to_set_density has not been called");
  *count = 0;
  if (c->dim != 3) return TO_OK;
  cudaStream_t s = c->stream;
  to_status st;
  if (c->hier_stale && (st = build_hierarchy(c)) != TO_OK) return st;
  int dev = 0;
  CUDA_TRY(c, cudaGetDevice(&dev), "device");
  // the launches as the solver makes them, on scratch buffers
  const int t = mg_t(c);
  auto args_of = [&](int kind, ApplyArgs* a) -> bool {
    LevelBuf* lv = c->lv;
    switch (kind) {
      case TO_TUNE_OP_APPLY:
        *a = c->mixed ? fine_args(c, TO_OP_K, T_F32, T_F32, T_F32, c->p32, c->q32, nullptr, nullptr,
                                  EPI_APPLY)
                      : fine_args(c, TO_OP_K, T_F64, T_F64, T_F64, c->p, c->q, nullptr, nullptr,
                                  EPI_APPLY);
        a->clean_inputs = true;   // timed as the solver launches it (scratch values)
        return true;
      case TO_TUNE_OP_RESID:
      case TO_TUNE_OP_SMOOTH:
        *a = fine_args(c, TO_OP_K, t, t, t, lv[0].z, lv[0].r, lv[0].b, lv[0].dinv,
                       kind == TO_TUNE_OP_RESID ? EPI_RESID : EPI_SMOOTH);
        a->clean_inputs = true;
        return true;
      case TO_TUNE_GAL1_RESID:
      case TO_TUNE_GAL1_SMOOTH:
        if (!c->l1_implicit) return false;
        *a = coarse_args(c, 1, lv[1].z, kind == TO_TUNE_GAL1_RESID ? lv[1].r : lv[1].z2, lv[1].b,
                         kind == TO_TUNE_GAL1_RESID ? EPI_RESID : EPI_SMOOTH);
        a->clean_inputs = true;
        return true;
      case TO_TUNE_ACC_APPLY:
      case TO_TUNE_ACC_RESID:
        if (!(c->mixed && c->df_ok)) return false;
        *a = fine_args(c, TO_OP_K, T_DF, T_D2, T_D2, c->p, c->t,
                       kind == TO_TUNE_ACC_RESID ? c->fd : nullptr, nullptr,
                       kind == TO_TUNE_ACC_RESID ? EPI_RESID : EPI_APPLY);
        return true;
    }
    return false;
  };
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CUDA_TRY(c, cudaEventCreate(&e0), "event");
  CUDA_TRY(c, cudaEventCreate(&e1), "event");
  auto time_us = [&](const ApplyArgs& a, double* us) -> cudaError_t {
    cudaError_t e;
    for (int w = 0; w < 2; ++w)
      if ((e = launch_apply(a, s)) != cudaSuccess) return e;
    if ((e = cudaEventRecord(e0, s)) != cudaSuccess) return e;
    for (int r = 0; r < reps; ++r)
      if ((e = launch_apply(a, s)) != cudaSuccess) return e;
    if ((e = cudaEventRecord(e1, s)) != cudaSuccess) return e;
    if ((e = cudaEventSynchronize(e1)) != cudaSuccess) return e;
    float ms = 0.f;
    if ((e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) return e;
    *us = 1e3 * ms / reps;
    return cudaSuccess;
  };
  cudaError_t err = cudaSuccess;
  for (int kind = 0; kind < TO_TUNE_N && err == cudaSuccess; ++kind) {
    ApplyArgs a;
    if (!args_of(kind, &a)) continue;
    const auto key = std::make_tuple(dev * 64 + kind * 4 + (c->mixed ? 1 : 0) + (c->use_tc ? 2 : 0),
                                     kind,
                                     (long long)a.g.nnx, (long long)a.g.nny, (long long)a.g.nnz);
    to_tune_result r{kind, 0, 0, 0.0, 0.0, 0};
    {
      std::lock_guard<std::mutex> lock(g_tune_mu);
      auto it = g_tune_cache.find(key);
      if (it != g_tune_cache.end()) {
        c->tuned_zc[kind] = it->second.first;
        c->tuned_var[kind] = it->second.second;
        r.chunk_layers = it->second.first;
        r.variant = it->second.second;
        if (*count < cap) results[*count] = r;
        ++*count;
        continue;
      }
    }
    a.zsplit = 0;
    a.variant = 0;
    double h_us = 0.0;
    if ((err = time_us(a, &h_us)) != cudaSuccess) break;
    double best_us = h_us;
    int best = 0, best_var = 0, tried = 0;
    const int nnz = (int)a.g.nnz;
    // the pair kernel (float32 finest grid) also has a second register
    // variant (bit 0) and the work-list launch of either (bit 1)
    const bool pair = kind <= TO_TUNE_OP_SMOOTH && pair_apply_ok(a) && !a.use_tc;
    for (int var = 0; var <= (pair ? 3 : 0) && err == cudaSuccess; ++var) {
      for (int nzc = 1; nzc <= nnz && nzc <= 64; ++nzc) {
        const int zc = (nnz + nzc - 1) / nzc;
        if (zc < 2 || (nnz + zc - 1) / zc != nzc) continue;
        a.zsplit = zc;
        a.variant = var;
        double us = 0.0;
        if ((err = time_us(a, &us)) != cudaSuccess) break;
        ++tried;
        if (us < 0.99 * best_us) {
          best_us = us;
          best = zc;
          best_var = var;
        }
      }
    }
    if (err != cudaSuccess) break;
    c->tuned_zc[kind] = best;
    c->tuned_var[kind] = best_var;
    {
      std::lock_guard<std::mutex> lock(g_tune_mu);
      g_tune_cache[key] = std::make_pair(best, best_var);
    }
    r.candidates = tried;
    r.chunk_layers = best;
    r.variant = best_var;
    r.chosen_us = best_us;
    r.heuristic_us = h_us;
    if (*count < cap) results[*count] = r;
    ++*count;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != cudaSuccess) return cuda_fail(c, "autotune", err);
  // captured V-cycles carry the old launch shapes
  for (int q = 0; q < c->n_vgraph; ++q) cudaGraphExecDestroy(c->vgraph[q].exec);
  c->n_vgraph = 0;
  return TO_OK;
}

to_status to_operator_options(to_ctx* c, int32_t flags) {
  if (!c) return fail(c, TO_E_INVALID, "NULL argument");
  if (flags & ~(TO_OPERATOR_TENSOR_CORES | TO_OPERATOR_FUSED_COARSE | TO_OPERATOR_TALL_TILES |
                TO_OPERATOR_WORK_LIST))
    return fail(c, TO_E_INVALID, "unknown operator option");
  const bool tc = (flags & TO_OPERATOR_TENSOR_CORES) != 0;
  const bool fuse = (flags & TO_OPERATOR_FUSED_COARSE) != 0;
  const bool tall = (flags & TO_OPERATOR_TALL_TILES) != 0;
  const bool wl = (flags & TO_OPERATOR_WORK_LIST) != 0;
  if (tall != c->tall_tiles || wl != c->work_list) {
    c->tall_tiles = tall;
    c->work_list = wl;
    for (int q = 0; q < c->n_vgraph; ++q) cudaGraphExecDestroy(c->vgraph[q].exec);
    c->n_vgraph = 0;   // recaptured with the selected tile
  }
  if (tc && !c->tc_bmat) return fail(c, TO_E_INVALID, "the tensor-core operator is 3D only");
  if (tc != c->use_tc || fuse != c->fuse_coarse) {
    if (tc != c->use_tc)
      for (int q = 0; q < 8; ++q) c->tuned_zc[q] = c->tuned_var[q] = 0;
    c->use_tc = tc;
    c->fuse_coarse = fuse;
    for (int q = 0; q < c->n_vgraph; ++q) cudaGraphExecDestroy(c->vgraph[q].exec);
    c->n_vgraph = 0;   // recaptured with the selected kernels
  }
  return TO_OK;
}

to_status to_carm_options(to_ctx* c, int32_t flags) {
  if (!c) return fail(c, TO_E_INVALID, "NULL argument");
  if (flags & ~TO_CARM_R1_PROJECTED_LOAD) return fail(c, TO_E_INVALID, "unknown CARM option");
  c->carm_flags = flags;
  return TO_OK;
}

to_status to_carm_info(to_ctx* c, int32_t* kq, int32_t* k, double* sigma) {
  if (!c || !kq || !k) return fail(c, TO_E_INVALID, "NULL argument");
  if (c->carm_built < 1) return fail(c, TO_E_STATE, "to_carm_build has not been called");
  *kq = c->carm_qr;
  *k = c->carm_built;
  if (sigma) {
    CUDA_TRY(c, cudaMemcpyAsync(sigma, c->small + SM_SIG, sizeof(double) * c->desc.n_carm,
                                cudaMemcpyDeviceToHost, c->stream), "read sigma");
    CUDA_TRY(c, cudaStreamSynchronize(c->stream), "sync");
  }
  return TO_OK;
}

to_status to_carm_basis_column(to_ctx* c, int32_t j, double* out) {
  if (!c || !out) return fail(c, TO_E_INVALID, "NULL argument");
  if (c->carm_built < 1) return fail(c, TO_E_STATE, "to_carm_build has not been called");
  if (j < 0 || j >= c->carm_built) return fail(c, TO_E_INVALID, "column index out of range");
  LAUNCH(c, launch_vconvert(c->n, vt(c), c->R + (size_t)j * c->n, V_F64, out, c->stream),
         "basis column");
  return TO_OK;
}

to_status to_carm_basis_error(to_ctx* c, double* err) {
  if (!c || !err) return fail(c, TO_E_INVALID, "NULL argument");
  if (c->carm_built < 1) return fail(c, TO_E_STATE, "to_carm_build has not been called");
  const int k = c->carm_built;
  LAUNCH(c, launch_gram_sym(c->n, vt(c), c->R, c->R, k, c->small + SM_KR, k, c->partials,
                            c->counters + C_MULTI, c->stream), "basis Gram");
  std::vector<double> G((size_t)k * k);
  CUDA_TRY(c, cudaMemcpyAsync(G.data(), c->small + SM_KR, sizeof(double) * k * k,
                              cudaMemcpyDeviceToHost, c->stream), "read");
  CUDA_TRY(c, cudaStreamSynchronize(c->stream), "sync");
  double e = 0.0;
  for (int j = 0; j < k; ++j)
    for (int i = 0; i < k; ++i) e = std::max(e, fabs(G[i + (size_t)k * j] - (i == j ? 1.0 : 0.0)));
  *err = e;
  return TO_OK;
}

to_status to_carm_solve(to_ctx* c, double* u, double* eps, double* eps_dev) {
  if (!c || !u) return fail(c, TO_E_INVALID, "NULL argument");
  if (c->carm_built < 1) return fail(c, TO_E_STATE, "to_carm_build has not been called");
  cudaStream_t s = c->stream;
  const long long n = c->n;
  const int k = c->carm_built;
  to_status st;
  double* small = c->small;
  const int v = vt(c);
  const double* fv = c->mixed ? c->fd : c->f;
  // K R~ enters the reduced matrix and the residual check, so it always uses
  // the float64-accurate operator; the basis itself may be built in float32.
  for (int j = 0; j < k; ++j)
    if ((st = apply_accurate_vec(c, TO_OP_K, c->R + (size_t)j * n, c->Q + (size_t)j * n,
                                 EPI_APPLY)) != TO_OK)
      return st;
  LAUNCH(c, launch_gram_sym(n, v, c->R, c->Q, k, small + SM_KR, k, c->partials,
                            c->counters + C_MULTI, s), "K_R");
  LAUNCH(c, launch_gram(n, v, c->R, k, nullptr, fv, 1, nullptr, small + SM_FR, k, c->partials,
                        c->counters + C_MULTI, s), "f_R");
  LAUNCH(c, launch_small_chol_solve(k, nullptr, small + SM_KR, small + SM_FR, small + SM_Y,
                                    c->ints + I_STATUS, s), "K_R y = f_R");
  LAUNCH(c, launch_combine(n, v, c->R, k, nullptr, small + SM_Y, 1.0, 0.0, u, V_F64, nullptr,
                           nullptr, c->partials, c->counters + C_UPD, s), "u = R y");
  LAUNCH(c, launch_combine(n, v, c->Q, k, nullptr, small + SM_Y, 1.0, 0.0, c->t, v, fv,
                           c->scal + S_RR, c->partials, c->counters + C_UPD, s), "K R y - f");
  LAUNCH(c, launch_eps(c->scal, S_RR, S_FNORM2, c->scal + S_EPS, s), "eps");
  if (eps_dev)
    CUDA_TRY(c, cudaMemcpyAsync(eps_dev, c->scal + S_EPS, 8, cudaMemcpyDeviceToDevice, s), "eps");
  if (eps) {
    if ((st = read_scalar(c, c->scal + S_EPS, eps)) != TO_OK) return st;
  }
  return TO_OK;
}

to_status to_sensitivity(to_ctx* c, const double* u, double* compliance_dev, double* dc) {
  if (!c || !u || !compliance_dev || !dc) return fail(c, TO_E_INVALID, "NULL argument");
  if (!c->have_density) return fail(c, TO_E_STATE, "to_set_density has not been called");
  const to_mesh_desc& d = c->desc;
  // mixed path: double-float arithmetic on the FP32 pipe (float64 otherwise)
  if (c->mixed && sensitivity_df_ok(c->dim, d.penal))
    LAUNCH(c, launch_sensitivity_df(c->lv[0].g, c->lv[0].mask, c->wht64, u, c->E64, c->rho_phys,
                                    d.penal, d.E0, d.Emin, dc, compliance_dev, c->partials,
                                    c->counters + C_SENS, c->stream), "sensitivity");
  else
    LAUNCH(c, launch_sensitivity(c->dim, c->lv[0].g, c->lv[0].mask, c->KE64,
                                 c->dim == 3 ? c->wht64 : nullptr, u, c->E64,
                                 c->rho_phys, d.penal, d.E0, d.Emin, dc, compliance_dev,
                                 c->partials, c->counters + C_SENS, c->stream), "sensitivity");
  return TO_OK;
}

to_status to_mesh_springs(to_ctx* c, int32_t n, const int64_t* dofs, const double* k) {
  if (!c || n < 0 || (n > 0 && (!dofs || !k))) return fail(c, TO_E_INVALID, "bad arguments");
  if (c->dim != 2) return fail(c, TO_E_INVALID, "springs are supported on 2D grids");
  if (n > TO_MAX_SPRINGS) return fail(c, TO_E_INVALID, "too many springs");
  Springs sp;
  sp.n = n;
  for (int q = 0; q < n; ++q) {
    if (dofs[q] < 0 || dofs[q] >= c->n) return fail(c, TO_E_INVALID, "spring DOF out of range");
    if (!(k[q] >= 0.0) || !std::isfinite(k[q])) return fail(c, TO_E_INVALID, "bad spring stiffness");
    for (int r = 0; r < q; ++r)
      if (dofs[r] == dofs[q]) return fail(c, TO_E_INVALID, "spring DOF repeated");
    uint8_t m = 0;
    CUDA_TRY(c, cudaMemcpyAsync(&m, c->lv[0].mask + dofs[q] / c->dim, 1, cudaMemcpyDeviceToHost,
                                c->stream), "read mask");
    CUDA_TRY(c, cudaStreamSynchronize(c->stream), "sync");
    if ((m >> (dofs[q] % c->dim)) & 1u) return fail(c, TO_E_INVALID, "spring on a fixed DOF");
    sp.dof[q] = dofs[q];
    sp.k[q] = k[q];
  }
  c->springs = sp;
  c->hier_stale = true;   // diagonal and level-1 matrices include the springs
  for (int q = 0; q < c->n_vgraph; ++q) cudaGraphExecDestroy(c->vgraph[q].exec);
  c->n_vgraph = 0;        // captured launches carry the old springs
  return TO_OK;
}

to_status to_sensitivity_adjoint(to_ctx* c, const double* u, const double* lam,
                                 double* mutual_dev, double* dc) {
  if (!c || !u || !lam || !mutual_dev || !dc) return fail(c, TO_E_INVALID, "NULL argument");
  if (!c->have_density) return fail(c, TO_E_STATE, "to_set_density has not been called");
  const to_mesh_desc& d = c->desc;
  LAUNCH(c, launch_sensitivity(c->dim, c->lv[0].g, c->lv[0].mask, c->KE64, nullptr, u, c->E64,
                               c->rho_phys, d.penal, d.E0, d.Emin, dc, mutual_dev, c->partials,
                               c->counters + C_SENS, c->stream, lam), "adjoint sensitivity");
  return TO_OK;
}

to_status to_oc_options(to_ctx* c, double eta) {
  if (!c) return fail(c, TO_E_INVALID, "NULL argument");
  if (!(eta > 0.0 && eta <= 1.0)) return fail(c, TO_E_INVALID, "eta must be in (0, 1]");
  c->oc_eta = eta;
  return TO_OK;
}

to_status to_filter(to_ctx* c, int32_t mode, const double* in, double* out) {
  if (!c || !in || !out || in == out) return fail(c, TO_E_INVALID, "bad arguments");
  if (mode != TO_FILTER_DENSITY && mode != TO_FILTER_SENS) return fail(c, TO_E_INVALID, "bad mode");
  LAUNCH(c, launch_filter(c->dim, c->lv[0].g, c->stencil, mode, c->invHs, in, out, c->stream),
         "filter");
  return TO_OK;
}

}  // extern "C"

// The OC update with a fixed number of lambda sections and no host read, so
// that it can be captured into a graph: a section is a no-op once the
// bracket is within 1e-13, and 48 sections cover the 7 geometric and ~16
// even cuts the search takes, so the result equals to_oc_update's.
to_status oc_update_enqueue(to_ctx* c, double volfrac, double move, const double* dc_f,
                            const double* dv_f, double* rho, double* change_dev) {
  cudaStream_t s = c->stream;
  const long long nel = c->nel;
  const double target = volfrac * (double)nel;
  LAUNCH(c, launch_oc_prep_d(nel, rho, dc_f, dv_f, move, c->oc_a, c->oc_a2, c->oc_lo, c->oc_hi,
                             c->oc_dv2, c->scal, s, c->oc_eta), "oc prep");
  for (int q = 0; q < 48; ++q)
    LAUNCH(c, launch_oc_section(nel, c->oc_a2, c->oc_lo, c->oc_hi, c->oc_dv2, target, c->scal,
                                c->partials, c->counters + C_OC, s, c->oc_eta), "oc section");
  LAUNCH(c, launch_oc_final(nel, rho, c->oc_a, move, c->scal, change_dev, c->partials,
                            c->counters + C_MAX, s, c->oc_eta), "oc final");
  return TO_OK;
}

extern "C" {

to_status to_oc_update(to_ctx* c, double volfrac, double move, const double* dc_f,
                       const double* dv_f, double* rho, double* change_dev) {
  if (!c || !dc_f || !dv_f || !rho) return fail(c, TO_E_INVALID, "NULL argument");
  if (!(volfrac > 0.0 && volfrac <= 1.0) || !(move > 0.0 && move <= 1.0))
    return fail(c, TO_E_INVALID, "bad volfrac/move");
  cudaStream_t s = c->stream;
  const long long nel = c->nel;
  const double target = volfrac * (double)nel;
  LAUNCH(c, launch_oc_prep_d(nel, rho, dc_f, dv_f, move, c->oc_a, c->oc_a2, c->oc_lo, c->oc_hi,
                             c->oc_dv2, c->scal, s, c->oc_eta), "oc prep");
  // eight-way sections run on the device; a launch is a no-op once the
  // bracket is within a relative 1e-13.  From [0, 1e9] geometric cuts reach
  // lambda's magnitude in a few sweeps (at most 7 for lambda >= 1e-40) and
  // 15 more evenly spaced cuts reach 1e-13, so 24 are queued before the
  // host first looks, then 8 at a time.
  for (int chunk = 0, nsec = 24; chunk < 16; ++chunk, nsec = 8) {
    for (int q = 0; q < nsec; ++q)
      LAUNCH(c, launch_oc_section(nel, c->oc_a2, c->oc_lo, c->oc_hi, c->oc_dv2, target, c->scal,
                                  c->partials, c->counters + C_OC, s, c->oc_eta), "oc section");
    double lr[2];
    CUDA_TRY(c, cudaMemcpyAsync(lr, c->scal + S_OC_L1, 16, cudaMemcpyDeviceToHost, s), "read");
    CUDA_TRY(c, cudaStreamSynchronize(s), "sync");
    if (!((lr[1] - lr[0]) > 1e-13 * (lr[0] + lr[1]))) break;
  }
  LAUNCH(c, launch_oc_final(nel, rho, c->oc_a, move, c->scal, change_dev, c->partials,
                            c->counters + C_MAX, s, c->oc_eta), "oc final");
  return TO_OK;
}

to_status to_profile_enable(to_ctx* c, int32_t kinds) {
  if (!c) return fail(c, TO_E_INVALID, "NULL ctx");
  if (kinds < 0 || kinds >= (1 << PK_N)) return fail(c, TO_E_INVALID, "bad kind mask");
  c->prof_mask = (unsigned)kinds;
  return TO_OK;
}

to_status to_profile_read(to_ctx* c, int32_t kind, int64_t* count, double* ms, double* bytes) {
  if (!c || !count || !ms || kind < 0 || kind >= PK_N) return fail(c, TO_E_INVALID, "bad arguments");
  CUDA_TRY(c, cudaStreamSynchronize(c->stream), "sync");
  int64_t cnt = 0;
  double tot = 0.0, byt = 0.0;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> keep;
  std::vector<double> keep_b;
  for (size_t q = 0; q < c->ev_used.size(); ++q) {
    auto& u = c->ev_used[q];
    if (u.first == kind) {
      float t = 0.0f;
      if (cudaEventElapsedTime(&t, u.second.first, u.second.second) == cudaSuccess) {
        tot += t;
        byt += c->ev_bytes[q];
        cnt++;
      }
      c->ev_pool.push_back(u.second.first);
      c->ev_pool.push_back(u.second.second);
    } else {
      keep.push_back(u);
      keep_b.push_back(c->ev_bytes[q]);
    }
  }
  c->ev_used.swap(keep);
  c->ev_bytes.swap(keep_b);
  *count = cnt;
  *ms = tot;
  if (bytes) *bytes = byt;
  return TO_OK;
}

to_status to_launch_count(to_ctx* c, int64_t* count, int32_t reset) {
  if (!c || !count) return fail(c, TO_E_INVALID, "bad arguments");
  *count = c->launches;
  if (reset) c->launches = 0;
  return TO_OK;
}

}  // extern "C"
