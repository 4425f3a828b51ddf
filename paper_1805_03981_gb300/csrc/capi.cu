// C ABI of the solver (include/dg.h): contexts, validation, dispatch and the
// time-stepping drivers.  All arithmetic of the hot path runs in the kernels
// of dg_kernels.cuh and setup.cu; this file only moves pointers and sizes.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/dg.h"
#include "dg_internal.h"
#include "dg2d.cuh"

using namespace dg;

namespace {

// Five-stage fourth-order 2N-storage Runge-Kutta (Carpenter & Kennedy, 1994).
const double kLsrkA[5] = {0.0, -567301805773.0 / 1357537059087.0,
                          -2404267990393.0 / 2016746695238.0,
                          -3550918686646.0 / 2091501179385.0,
                          -1275806237668.0 / 842570457699.0};
const double kLsrkB[5] = {1432997174477.0 / 9575080441755.0,
                          5161836677717.0 / 13612068292357.0,
                          1720146321549.0 / 2090206949498.0,
                          3134564353537.0 / 4481467310338.0,
                          2277821191437.0 / 14882151754819.0};

// The paper's two-register schemes (Sec. 2.2; Kennedy, Carpenter & Lewis
// 2000): LSRK4(5) = RK4(3)5[2R+]C and LSRK5(9) = RK5(4)9[2R+]S.  A[i] weights
// the newest increment in stage i+1, B[i] the increments of the solution.
const double kKcl45A[4] = {970286171893.0 / 4311952581923.0, 6584761158862.0 / 12103376702013.0,
                           2251764453980.0 / 15575788980749.0, 26877169314380.0 / 34165994151039.0};
const double kKcl45B[5] = {1153189308089.0 / 22510343858157.0, 1772645290293.0 / 4653164025191.0,
                           -1672844663538.0 / 4480602732383.0, 2114624349019.0 / 3568978502595.0,
                           5198255086312.0 / 14908931495163.0};
const double kKcl59A[8] = {1107026461565.0 / 5417078080134.0,   38141181049399.0 / 41724347789894.0,
                           493273079041.0 / 11940823631197.0,   1851571280403.0 / 6147804934346.0,
                           11782306865191.0 / 62590030070788.0, 9452544825720.0 / 13648368537481.0,
                           4435885630781.0 / 26285702406235.0,  2357909744247.0 / 11371140753790.0};
const double kKcl59B[9] = {2274579626619.0 / 23610510767302.0,  693987741272.0 / 12394497460941.0,
                           -347131529483.0 / 15096185902911.0,  1144057200723.0 / 32081666971178.0,
                           1562491064753.0 / 11797114684756.0,  13113619727965.0 / 44346030145118.0,
                           393957816125.0 / 7825732611452.0,    720647959663.0 / 6565743875477.0,
                           3559252274877.0 / 14424734981077.0};

std::mutex g_mu;
KernelTable g_kt;
KernelTable2D g_kt2;
bool g_kt_ready = false;
HostTables g_tab;
float g_tab_f[DG_TAB_LEN];
unsigned long long g_dev_ready = 0;  // bit per device with uploaded tables
thread_local std::string g_setup_err;

int init_device(int dev, std::string* err) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_kt_ready) {
    std::memset(&g_kt, 0, sizeof(g_kt));
    build_tables(&g_tab);
    for (int i = 0; i < DG_TAB_LEN; ++i) g_tab_f[i] = (float)g_tab.tab[i];
    register_f64_lo(&g_kt);
    register_f64_hi(&g_kt);
    register_f32_lo(&g_kt);
    register_f32_hi(&g_kt);
    register_tck_odd_f64(&g_kt);
    register_tck_odd_f32(&g_kt);
    register_tckc_f64_lo(&g_kt);
    register_tckc_f64_hi(&g_kt);
    register_tckc_f32_lo(&g_kt);
    register_tckc_f32_hi(&g_kt);
    register_tckn(&g_kt);
    register_tcki_f32(&g_kt);
    register_lsrk2r_f64(&g_kt);
    register_lsrk2r_f32(&g_kt);
    register_2d(&g_kt2);
    g_kt_ready = true;
  }
  if (dev < 0 || dev >= 64) {
    *err = "device index out of range";
    return DG_EINVAL;
  }
  if (!(g_dev_ready >> dev & 1ull)) {
    int (*up[])(const double*, const float*) = {
        upload_f64_lo,      upload_f64_hi,      upload_f32_lo,      upload_f32_hi,      upload_batch_f64,
        upload_batch_f32,   upload_tck_odd_f64, upload_tck_odd_f32, upload_tckc_f64_lo, upload_tckc_f64_hi,
        upload_tckc_f32_lo, upload_tckc_f32_hi, upload_tckn,        upload_lsrk2r_f64,  upload_lsrk2r_f32,
        upload_tcki_f32,    upload_2d};
    for (size_t i = 0; i < sizeof(up) / sizeof(up[0]); ++i) {
      const int e = up[i](g_tab.tab, g_tab_f);
      if (e) {
        cudaGetLastError();
        *err = std::string("kernel set-up (constant tables / shared memory limits) failed: ") +
               cudaGetErrorString((cudaError_t)e);
        return DG_ECUDA;
      }
    }
    g_dev_ready |= 1ull << dev;
  }
  return DG_OK;
}

}  // namespace

struct dg_ctx {
  int dev = 0;
  int E = 0, k = 0, n = 0, q = 0, prec = 0;
  int Erun = 0;  // elements stepped: the first Erun (the rest are ghosts of a partition)
  int dim = 3;   // 2: quadrilaterals (dg_mesh_setup_2d), state [E][3][n^2], Gauss basis inside the steppers
  double alpha = 1.0;
  size_t rsize = 8;
  int32_t* nbr = nullptr;
  int8_t* nbr_face = nullptr;
  int8_t* orient = nullptr;
  double* nodes = nullptr;
  double* rho = nullptr;
  double* c = nullptr;
  double* pts = nullptr;
  double* xq = nullptr;
  int* bad = nullptr;
  void* geoA = nullptr;
  void* geoM = nullptr;
  void* geoF = nullptr;
  void* geoT = nullptr;
  void* geoK = nullptr;   // compact affine data (affine meshes only)
  void* geoKT = nullptr;
  bool geo_affine = false;  // every element is an affine image of the cube
  bool affine = false;      // ... and has constant coefficients: compact kernels
  int tstride = 0;
  int tstep = 2;  // predictor geometry at Gauss sets n, n - tstep, ... (1 once a step reduces by 1 or 3)
  void* U2 = nullptr;    // LSRK intermediate stage states
  void* U3 = nullptr;
  void* dU = nullptr;    // LSRK register
  void* Ubar = nullptr;  // ADER predictor
  void* Wd = nullptr;    // HDG-ADER: the DG derivative of the state
  void* Uh = nullptr;    // state for dg_solve_host
  double* partial = nullptr;
  int partial_cap = 0;
  size_t dev_bytes = 0;
  uint64_t launches = 0;
  int epb_op = 1, epb_tck = 1, epb_en = 1;
  int expire_wait = 0;  // dg_test_expire_waits
  int lsrk_scheme = DG_LSRK_CK54;  // dg_set_lsrk_scheme
  int basis = DG_BASIS_GL;  // representation of the state inside the steppers
  int pred_kernel = DG_PRED_AUTO;  // predictor kernel for Gauss-point states
  // profiling: event pairs recorded around launches while enabled
  bool prof = false;
  struct Rec {
    int kind;
    cudaEvent_t a, b;
  };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> event_pool;
  std::vector<void*> allocs;
  std::string err;

  int npts() const { return dim == 2 ? n * n : n * n * n; }  // nodes per element
  size_t state_elems() const { return (size_t)E * (dim + 1) * npts(); }
  size_t run_elems() const { return (size_t)Erun * (dim + 1) * npts(); }
  size_t state_bytes() const { return state_elems() * rsize; }

  int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    err = buf;
    return code;
  }
  int cuda_fail(cudaError_t e, const char* what) {
    return fail(DG_ECUDA, "%s: %s", what, cudaGetErrorString(e));
  }
  template <typename T>
  int alloc(T** p, size_t bytes, const char* what) {
    void* v = nullptr;
    cudaError_t e = cudaMalloc(&v, bytes ? bytes : 16);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(DG_ENOMEM, "cudaMalloc(%zu) for %s failed: %s", bytes, what, cudaGetErrorString(e));
    }
    allocs.push_back(v);
    dev_bytes += bytes;
    *p = static_cast<T*>(v);
    return DG_OK;
  }
  void release(void* p, size_t bytes) {
    for (size_t i = 0; i < allocs.size(); ++i)
      if (allocs[i] == p) {
        cudaFree(p);
        allocs.erase(allocs.begin() + i);
        dev_bytes -= bytes;
        return;
      }
  }
  cudaEvent_t take_event() {
    if (!event_pool.empty()) {
      cudaEvent_t ev = event_pool.back();
      event_pool.pop_back();
      return ev;
    }
    cudaEvent_t ev = nullptr;
    if (cudaEventCreate(&ev) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return ev;
  }
  // bracket one launch with events when profiling is on
  struct Span {
    dg_ctx* c;
    int kind;
    cudaStream_t st;
    cudaEvent_t a = nullptr;
    Span(dg_ctx* c_, int k, cudaStream_t s) : c(c_), kind(k), st(s) {
      if (c->prof && (a = c->take_event())) cudaEventRecord(a, st);
    }
    void done() {
      if (!a) return;
      cudaEvent_t b = c->take_event();
      if (b) {
        cudaEventRecord(b, st);
        c->recs.push_back({kind, a, b});
      } else {
        c->event_pool.push_back(a);
      }
      a = nullptr;
    }
  };
  ~dg_ctx() {
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(dev);
    for (auto& r : recs) {
      cudaEventDestroy(r.a);
      cudaEventDestroy(r.b);
    }
    for (auto ev : event_pool) cudaEventDestroy(ev);
    for (void* p : allocs) cudaFree(p);
    cudaSetDevice(cur);
  }
};

namespace {

#define DG_CK(call, what)                              \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return ctx->cuda_fail(e_, what); \
  } while (0)

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

inline cudaStream_t S(uintptr_t s) { return reinterpret_cast<cudaStream_t>(s); }

// the 2D path (defined with dg_mesh_setup_2d below)
int run_setup2(dg_ctx* ctx, cudaStream_t st);
int change_basis2(dg_ctx* ctx, void* U, int to_g, cudaStream_t st);
int lsrk_steps2(dg_ctx* ctx, void* U, double dt, int nsteps, cudaStream_t st);
int ader_steps2(dg_ctx* ctx, void* U, double dt, int nsteps, int red, cudaStream_t st);
int apply2(dg_ctx* ctx, const void* U, void* R, cudaStream_t st);
int tck2_gl(dg_ctx* ctx, const void* U, void* Ubar, double dt, int red, cudaStream_t st);
int energy2(dg_ctx* ctx, const void* U, double* out, cudaStream_t st);

int orient_map(int o, int n, int i, int j, int* ip, int* jp) {
  const int u = (o & 1) ? j : i, v = (o & 1) ? i : j;
  *ip = (o & 2) ? n - 1 - u : u;
  *jp = (o & 4) ? n - 1 - v : v;
  return 0;
}

int validate_mesh(const dg_mesh_desc* m, std::string* err) {
  char buf[256];
  const int E = m->n_elem;
  for (int e = 0; e < E; ++e)
    for (int f = 0; f < 6; ++f) {
      const int en = m->nbr[e * 6 + f];
      if (en < -1 || en >= E) {
        snprintf(buf, sizeof buf, "nbr[%d][%d] = %d out of range", e, f, en);
        *err = buf;
        return DG_EMESH;
      }
      if (en < 0) continue;
      const int fn = m->nbr_face[e * 6 + f], o = m->orient[e * 6 + f];
      if (fn < 0 || fn >= 6 || o < 0 || o >= 8) {
        snprintf(buf, sizeof buf, "nbr_face/orient of (%d,%d) out of range", e, f);
        *err = buf;
        return DG_EMESH;
      }
      if (m->nbr[en * 6 + fn] != e || m->nbr_face[en * 6 + fn] != f) {
        snprintf(buf, sizeof buf, "face (%d,%d) -> (%d,%d) is not reciprocated", e, f, en, fn);
        *err = buf;
        return DG_EMESH;
      }
      const int ob = m->orient[en * 6 + fn];
      if (ob < 0 || ob >= 8) {
        *err = "orient out of range";
        return DG_EMESH;
      }
      for (int j = 0; j < 3; ++j)
        for (int i = 0; i < 3; ++i) {
          int i1, j1, i2, j2;
          orient_map(o, 3, i, j, &i1, &j1);
          orient_map(ob, 3, i1, j1, &i2, &j2);
          if (i2 != i || j2 != j) {
            snprintf(buf, sizeof buf, "orientation codes of face (%d,%d) and (%d,%d) are not inverse",
                     e, f, en, fn);
            *err = buf;
            return DG_EMESH;
          }
        }
    }
  return DG_OK;
}

// Is every element the affine image of the reference cube?  The geometry
// nodes must lie on the affine map through the corners (-1,-1,-1), (+1,-1,-1),
// (-1,+1,-1), (-1,-1,+1).
bool mesh_is_affine(const dg_mesh_desc* m) {
  const int q = m->geom_degree, c = q + 1;
  std::vector<double> xq(DG_NMAX + 2);
  gauss_lobatto(c, xq.data());
  for (int e = 0; e < m->n_elem; ++e) {
    const double* X = m->nodes + (size_t)e * c * c * c * 3;
    auto node = [&](int i, int j, int k) { return X + 3 * (i + c * j + c * c * k); };
    const double *x0 = node(0, 0, 0), *xa = node(q, 0, 0), *xb = node(0, q, 0), *xc = node(0, 0, q);
    double scale = 0.0;
    for (int d = 0; d < 3; ++d)
      scale = std::max(scale, std::fabs(xa[d] - x0[d]) + std::fabs(xb[d] - x0[d]) + std::fabs(xc[d] - x0[d]));
    for (int k = 0; k < c; ++k)
      for (int j = 0; j < c; ++j)
        for (int i = 0; i < c; ++i) {
          const double* y = node(i, j, k);
          const double s = 0.5 * (xq[i] + 1), t = 0.5 * (xq[j] + 1), u = 0.5 * (xq[k] + 1);
          for (int d = 0; d < 3; ++d) {
            const double aff = x0[d] + s * (xa[d] - x0[d]) + t * (xb[d] - x0[d]) + u * (xc[d] - x0[d]);
            if (std::fabs(y[d] - aff) > 1e-12 * scale) return false;
          }
        }
  }
  return true;
}

// Are the nodal coefficient values constant within every element?
bool coef_constant(const double* rho, const double* c, int E, int n3) {
  if (!rho) return true;
  for (int e = 0; e < E; ++e)
    for (int i = 1; i < n3; ++i) {
      const size_t a = (size_t)e * n3, b = a + i;
      if (rho[b] != rho[a] || c[b] != c[a]) return false;
    }
  return true;
}

int pick_epb(int n, int bytes_per_elem, int target_threads, int max_threads) {
  int epb = target_threads / (n * n);
  if (epb < 1) epb = 1;
  const int smem_lim = 200 * 1024;
  while (epb > 1 && (epb * bytes_per_elem > smem_lim || epb * n * n > max_threads)) --epb;
  return epb;
}

int run_setup(dg_ctx* ctx, cudaStream_t st) {
  if (ctx->dim == 2) return run_setup2(ctx, st);
  SetupParams P;
  P.E = ctx->E;
  P.n = ctx->n;
  P.q = ctx->q;
  P.alpha = ctx->alpha;
  P.nodes = ctx->nodes;
  P.rho = ctx->rho;
  P.c = ctx->c;
  P.nbr = ctx->nbr;
  P.nbr_face = ctx->nbr_face;
  P.orient = ctx->orient;
  P.pts = ctx->pts;
  P.xq = ctx->xq;
  P.geoA = ctx->geoA;
  P.geoM = ctx->geoM;
  P.geoF = ctx->geoF;
  P.geoT = ctx->geoT;
  P.geoK = ctx->affine ? ctx->geoK : nullptr;
  P.geoKT = ctx->affine ? ctx->geoKT : nullptr;
  P.tstride = ctx->tstride;
  P.tstep = ctx->tstep;
  P.prec = ctx->prec;
  P.bad = ctx->bad;
  DG_CK(cudaMemsetAsync(ctx->bad, 0, sizeof(int), st), "memset");
  DG_CK(launch_setup(P, st), "setup kernel launch");
  ctx->launches++;
  int bad = 0;
  DG_CK(cudaMemcpyAsync(&bad, ctx->bad, sizeof(int), cudaMemcpyDeviceToHost, st), "copy flag");
  DG_CK(cudaStreamSynchronize(st), "setup kernel");
  if (bad) return ctx->fail(DG_EMESH, "non-positive Jacobian determinant in the mesh");
  return DG_OK;
}

OpParams op_params(const dg_ctx* ctx) {
  OpParams p;
  std::memset(&p, 0, sizeof(p));
  p.nbr = ctx->nbr;
  p.nbr_face = ctx->nbr_face;
  p.orient = ctx->orient;
  p.geoA = ctx->geoA;
  p.geoM = ctx->geoM;
  p.geoF = ctx->geoF;
  p.geoK = ctx->geoK;
  p.err = ctx->bad;
  p.E = ctx->Erun;
  p.expire_wait = ctx->expire_wait;
  return p;
}

int launch_op(dg_ctx* ctx, const OpParams& p, int epi, cudaStream_t st, bool gbasis = false) {
  OpFn fn = gbasis ? (ctx->affine ? g_kt.opga[ctx->prec][ctx->n] : g_kt.opg[ctx->prec][ctx->n])
                   : g_kt.op[ctx->prec][ctx->n];
  const int kind = epi == EPI_WRITE ? DG_KIND_OPERATOR : (epi == EPI_LSRK ? DG_KIND_LSRK : DG_KIND_ADER);
  dg_ctx::Span span(ctx, kind, st);
  DG_CK(fn(p, epi, ctx->epb_op, st), "operator kernel launch");
  span.done();
  ctx->launches++;
  return DG_OK;
}

// In-place change of basis of a whole state (GL <-> G).
int change_basis(dg_ctx* ctx, void* U, int to_g, cudaStream_t st) {
  if (ctx->dim == 2) return change_basis2(ctx, U, to_g, st);
  dg_ctx::Span span(ctx, DG_KIND_OTHER, st);
  DG_CK(g_kt.basis[ctx->prec][ctx->n](U, U, ctx->Erun, to_g, ctx->epb_en, st), "basis kernel launch");
  span.done();
  ctx->launches++;
  return DG_OK;
}

// Predictor kernel for Gauss-point states (dg_set_predictor_kernel).  By
// default FP32 takes the column form, which issues fewer shared-memory and
// index instructions; FP64 takes the line form, whose block-wide spreading
// keeps every lane of the FP64 pipe busy at the reduced Gauss sets.
bool use_columns(const dg_ctx* ctx) {
  if (ctx->pred_kernel == DG_PRED_LINES || g_kt.tckc[ctx->prec][ctx->n] == nullptr) return false;
  return ctx->pred_kernel == DG_PRED_COLUMNS || ctx->pred_kernel == DG_PRED_INTERLEAVED || ctx->prec == DG_FP32;
}

// The interleaved column form (affine elements with constant coefficients,
// Gauss-point states, reduction every 0 or 2 derivatives, no HDG derivative,
// FP32): the default there, or chosen with DG_PRED_INTERLEAVED.  Its results
// are those of the column form up to rounding.
bool use_interleaved(const dg_ctx* ctx, int red, const void* W) {
  if (ctx->pred_kernel != DG_PRED_AUTO && ctx->pred_kernel != DG_PRED_INTERLEAVED) return false;
  return ctx->affine && ctx->dim == 3 && (red == 0 || red == 2) && W == nullptr &&
         g_kt.tcki[ctx->prec][ctx->n] != nullptr;
}

int launch_tck(dg_ctx* ctx, const void* U, void* Ubar, double dt, int red, cudaStream_t st,
               bool gbasis = false, const void* W = nullptr) {
  TckParams p;
  std::memset(&p, 0, sizeof(p));
  p.W = W;
  p.gmode = gbasis ? 1 : 0;
  p.aff = ctx->affine ? 1 : 0;
  p.geoKT = ctx->geoKT;
  p.U = U;
  p.Ubar = Ubar;
  p.geoT = ctx->geoT;
  p.geoT_stride = ctx->tstride;
  p.geo_step = ctx->tstep;
  p.E = ctx->Erun;
  p.err = ctx->bad;
  double fact = 1.0;
  for (int j = 0; j <= ctx->n; ++j) {  // dt^{j+1} / (j+1)!
    fact *= (j + 1);
    p.coef[j] = std::pow(dt, j + 1) / fact;
  }
  const bool odd = red == 1 || red == 3;
  const bool col = gbasis && use_columns(ctx);
  int epb = ctx->epb_tck;
  const int n2 = ctx->n * ctx->n;
  if (ctx->pred_kernel == DG_PRED_GL_PROJECTION) {  // Alg. 1: GL states, no reduction
    if (gbasis || red != 0 || W)
      return ctx->fail(DG_EUNSUPPORTED,
                       "the GL-projection predictor takes GL states, reduce_every 0 and no HDG derivative");
    const int per = g_kt.tckn_smem[ctx->prec][ctx->n](0);
    const int thr = g_kt.tckn_maxthr[ctx->prec][ctx->n]();
    while (epb > 1 && (epb * per > 200 * 1024 || epb * n2 > thr)) --epb;
    dg_ctx::Span span(ctx, DG_KIND_TCK, st);
    DG_CK(g_kt.tckn[ctx->prec][ctx->n](p, 0, epb, st), "predictor kernel launch");
    span.done();
    ctx->launches++;
    return DG_OK;
  }
  if (col && use_interleaved(ctx, red, W)) {
    dg_ctx::Span span(ctx, DG_KIND_TCK, st);
    DG_CK(g_kt.tcki[ctx->prec][ctx->n](p, red, 0, st), "predictor kernel launch");
    span.done();
    ctx->launches++;
    return DG_OK;
  }
  if (col) {
    const int per = g_kt.tckc_smem[ctx->prec][ctx->n](red);
    const int thr = g_kt.tckc_maxthr[ctx->prec][ctx->n]();
    while (epb > 1 && (epb * per > 200 * 1024 || epb * n2 > thr)) --epb;
  } else if (odd) {  // more accumulator levels: fewer elements may fit a block
    const int per = g_kt.smem[ctx->prec][ctx->n](1, red);
    const int thr = g_kt.tck_odd_maxthr[ctx->prec][ctx->n]();
    while (epb > 1 && (epb * per > 200 * 1024 || epb * n2 > thr)) --epb;
  }
  dg_ctx::Span span(ctx, DG_KIND_TCK, st);
  DG_CK((col ? g_kt.tckc : odd ? g_kt.tck_odd : g_kt.tck)[ctx->prec][ctx->n](p, red, epb, st),
        "predictor kernel launch");
  span.done();
  ctx->launches++;
  return DG_OK;
}

// Reduction every 1 or 3 derivatives visits Gauss sets that the default
// predictor geometry (sets n, n-2, ...) lacks: on first use, rebuild it at
// every set n, n-1, ..., 2 (curved or variable-coefficient meshes only; the
// compact affine data serves every set).
int ensure_levels(dg_ctx* ctx, int red, cudaStream_t st) {
  if ((red != 1 && red != 3) || ctx->tstep == 1 || ctx->affine || ctx->dim == 2) return DG_OK;
  const size_t old_bytes = (size_t)ctx->rsize * ctx->tstride * ctx->E;
  void* fresh = nullptr;
  const int stride1 = tck_geo_stride(ctx->n, 1);
  int rc = ctx->alloc(&fresh, (size_t)ctx->rsize * stride1 * ctx->E, "predictor geometry (every Gauss set)");
  if (rc) return rc;
  DG_CK(cudaStreamSynchronize(st), "predictor geometry rebuild");
  ctx->release(ctx->geoT, old_bytes);
  ctx->geoT = fresh;
  ctx->tstep = 1;
  ctx->tstride = stride1;
  return run_setup(ctx, st);
}

int check_red(dg_ctx* ctx, int red) {
  if (red < 0 || red > 3)
    return ctx->fail(DG_EUNSUPPORTED, "reduce_every must be 0, 1, 2 or 3 (got %d)", red);
  if (ctx->dim == 2 && red != 0 && red != 2)
    return ctx->fail(DG_EUNSUPPORTED, "2D meshes take reduce_every 0 or 2");
  return DG_OK;
}

int ensure(dg_ctx* ctx, void** p, const char* what) {
  if (*p) return DG_OK;
  return ctx->alloc(p, ctx->state_bytes(), what);
}

// The address under which kernels of the current device can read or write
// the host buffer h: its device view when h is pinned host memory mapped
// into the device's address space, h itself when it is managed memory;
// nullptr otherwise (pageable memory: the caller copies instead).  The view
// must be 16-byte aligned (the transfer kernels use vector accesses).
const void* device_view(const void* h) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, h) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  const void* v = nullptr;
  if (a.type == cudaMemoryTypeHost && a.devicePointer) v = a.devicePointer;
  if (a.type == cudaMemoryTypeManaged) v = h;
  if (v && reinterpret_cast<uintptr_t>(v) % 16 != 0) v = nullptr;
  return v;
}

int check_state_ptr(dg_ctx* ctx, const void* p, const char* what) {
  if (!p) return ctx->fail(DG_EINVAL, "%s is NULL", what);
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return ctx->fail(DG_EINVAL, "%s is not a device pointer", what);
  }
  if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
    return ctx->fail(DG_EINVAL, "%s is not device memory", what);
  if (a.type == cudaMemoryTypeDevice && a.device != ctx->dev)
    return ctx->fail(DG_EINVAL, "%s is memory of device %d, the context is on device %d", what, a.device,
                     ctx->dev);
  if (reinterpret_cast<uintptr_t>(p) % 16 != 0)  // bulk copies read states directly
    return ctx->fail(DG_EINVAL, "%s must be 16-byte aligned", what);
  return DG_OK;
}

// Stage s reads the state of stage s-1 and writes a different buffer
// (neighbours read face values of the input while it is being written):
// U -> A -> B -> A -> B -> U, so each step ends in U without a copy.
int lsrk2r_steps(dg_ctx* ctx, void* U, double dt, int nsteps, cudaStream_t st, bool keep_g);

// keep_g: U already holds Gauss-point values (Gauss-basis contexts) and keeps
// them on return; the caller changes basis (dg_solve_host fuses that change
// with its host transfers).
int lsrk_steps(dg_ctx* ctx, void* U, double dt, int nsteps, cudaStream_t st, bool keep_g = false) {
  if (ctx->dim == 2) return lsrk_steps2(ctx, U, dt, nsteps, st);
  if (ctx->lsrk_scheme != DG_LSRK_CK54) return lsrk2r_steps(ctx, U, dt, nsteps, st, keep_g);
  int rc;
  if ((rc = ensure(ctx, &ctx->U2, "LSRK state"))) return rc;
  if ((rc = ensure(ctx, &ctx->U3, "LSRK state"))) return rc;
  if ((rc = ensure(ctx, &ctx->dU, "LSRK register"))) return rc;
  OpParams p = op_params(ctx);
  const bool g = ctx->basis == DG_BASIS_G && nsteps > 0;
  if (g && !keep_g && (rc = change_basis(ctx, U, 1, st))) return rc;
  void* const chain[6] = {U, ctx->U2, ctx->U3, ctx->U2, ctx->U3, U};
  for (int s = 0; s < nsteps; ++s)
    for (int st5 = 0; st5 < 5; ++st5) {
      p.U = chain[st5];
      p.Uadd = chain[st5];
      p.out = chain[st5 + 1];
      p.dU = ctx->dU;
      p.cA = kLsrkA[st5];
      p.cB = kLsrkB[st5];
      p.dt = dt;
      p.first = st5 == 0;
      if ((rc = launch_op(ctx, p, EPI_LSRK, st, g))) return rc;
    }
  if (g && !keep_g && (rc = change_basis(ctx, U, 0, st))) return rc;
  return DG_OK;
}

// A stage of a two-register scheme: the operator kernel with the LSRK2R
// epilogue, at the largest tiling its instantiation can launch.
int launch_op2r(dg_ctx* ctx, const OpParams& p, cudaStream_t st, bool gbasis) {
  const int which = gbasis ? (ctx->affine ? 2 : 1) : 0;
  const int n2 = ctx->n * ctx->n;
  const int thr = g_kt.op2r_maxthr[ctx->prec][ctx->n]();
  int epb = ctx->epb_op;
  while (epb > 1 && epb * n2 > thr) --epb;
  dg_ctx::Span span(ctx, DG_KIND_LSRK, st);
  DG_CK(g_kt.op2r[ctx->prec][ctx->n](p, which, epb, st), "operator kernel launch");
  span.done();
  ctx->launches++;
  return DG_OK;
}

// The two-register schemes (Sec. 2.2): with S the running sum (ctx->dU),
// stage i reads its input Y_i and S_i and writes Y_{i+1} = S_i + dt A_i R(Y_i)
// and S_{i+1} = S_i + dt B_i R(Y_i).  Y_1 = S_1 = U, so the first stage reads
// S from the input itself; the stage inputs then alternate between U2 and U3
// (neighbours read a stage's input while it runs); the last stage writes the
// new solution S into U and no stage input.
int lsrk2r_steps(dg_ctx* ctx, void* U, double dt, int nsteps, cudaStream_t st, bool keep_g) {
  const double* A = ctx->lsrk_scheme == DG_LSRK45 ? kKcl45A : kKcl59A;
  const double* B = ctx->lsrk_scheme == DG_LSRK45 ? kKcl45B : kKcl59B;
  const int stages = ctx->lsrk_scheme == DG_LSRK45 ? 5 : 9;
  int rc;
  if ((rc = ensure(ctx, &ctx->U2, "LSRK state"))) return rc;
  if ((rc = ensure(ctx, &ctx->U3, "LSRK state"))) return rc;
  if ((rc = ensure(ctx, &ctx->dU, "LSRK running sum"))) return rc;
  OpParams p = op_params(ctx);
  const bool g = ctx->basis == DG_BASIS_G && nsteps > 0;
  if (g && !keep_g && (rc = change_basis(ctx, U, 1, st))) return rc;
  for (int s = 0; s < nsteps; ++s) {
    void* Y = U;
    for (int i = 0; i < stages; ++i) {
      void* next = (i % 2 == 0) ? ctx->U2 : ctx->U3;
      p.U = Y;
      p.first = i == 0;
      p.last = i == stages - 1;
      p.Uadd = i == 0 ? U : ctx->dU;
      p.dU = p.last ? U : ctx->dU;
      p.out = p.last ? nullptr : next;
      p.cA = p.last ? 0.0 : dt * A[i];
      p.cB = dt * B[i];
      p.dt = dt;
      if ((rc = launch_op2r(ctx, p, st, g))) return rc;
      Y = next;
    }
  }
  if (g && !keep_g && (rc = change_basis(ctx, U, 0, st))) return rc;
  return DG_OK;
}

// hdg: HDG-ADER (Eq. hdg-ader): each step first evaluates the DG derivative
// W = -M^-1 K U, which takes the place of the predictor's first term -S U.
int ader_steps(dg_ctx* ctx, void* U, double dt, int nsteps, int red, cudaStream_t st, bool hdg = false,
               bool keep_g = false) {
  if (ctx->dim == 2) {
    if (hdg) return ctx->fail(DG_EUNSUPPORTED, "HDG-ADER is not built for 2D meshes");
    return ader_steps2(ctx, U, dt, nsteps, red, st);
  }
  int rc;
  if ((rc = ensure(ctx, &ctx->Ubar, "ADER predictor"))) return rc;
  if (hdg && (rc = ensure(ctx, &ctx->Wd, "HDG-ADER derivative"))) return rc;
  OpParams p = op_params(ctx);
  const bool g = ctx->basis == DG_BASIS_G && nsteps > 0;
  if (g && !keep_g && (rc = change_basis(ctx, U, 1, st))) return rc;
  for (int s = 0; s < nsteps; ++s) {
    if (hdg) {
      OpParams q = op_params(ctx);
      q.U = U;
      q.out = ctx->Wd;
      if ((rc = launch_op(ctx, q, EPI_WRITE, st, g))) return rc;
    }
    if ((rc = launch_tck(ctx, U, ctx->Ubar, dt, red, st, g, hdg ? ctx->Wd : nullptr))) return rc;
    p.U = ctx->Ubar;
    p.Uadd = U;
    p.out = U;
    if ((rc = launch_op(ctx, p, EPI_ADD, st, g))) return rc;
  }
  if (g && !keep_g && (rc = change_basis(ctx, U, 0, st))) return rc;
  return DG_OK;
}

// Element-wise precision change of a state (checkpoint copies).
template <typename From, typename To>
__global__ void cast_kernel(const From* __restrict__ in, To* __restrict__ out, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = static_cast<To>(in[i]);
}

// Sums of squares with a fixed launch shape and summation order.
template <typename Real>
__global__ void sumsq_kernel(const Real* A, const Real* B, size_t n, double* part) {
  double saa = 0.0, sdd = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const double a = A[i];
    saa += a * a;
    if (B) {
      const double d = a - (double)B[i];
      sdd += d * d;
    }
  }
  __shared__ double r1[256], r2[256];
  r1[threadIdx.x] = saa;
  r2[threadIdx.x] = sdd;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      r1[threadIdx.x] += r1[threadIdx.x + w];
      r2[threadIdx.x] += r2[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = r1[0];
    part[2 * blockIdx.x + 1] = r2[0];
  }
}

// Both callers synchronise their stream after using the buffer, so an old,
// smaller buffer has no work in flight when it is released here.
int ensure_partial(dg_ctx* ctx, int n) {
  if (ctx->partial_cap >= n) return DG_OK;
  void* old = ctx->partial;
  const int old_cap = ctx->partial_cap;
  void* fresh = nullptr;
  int rc = ctx->alloc(&fresh, sizeof(double) * n, "partial sums");
  if (rc) return rc;
  if (old) ctx->release(old, sizeof(double) * old_cap);
  ctx->partial = static_cast<double*>(fresh);
  ctx->partial_cap = n;
  return DG_OK;
}

}  // namespace

extern "C" {

const char* dg_strerror(int s) {
  switch (s) {
    case DG_OK: return "ok";
    case DG_EINVAL: return "invalid argument";
    case DG_ENOMEM: return "out of memory";
    case DG_ECUDA: return "CUDA error";
    case DG_EUNSUPPORTED: return "unsupported";
    case DG_EAGAIN: return "not finished";
    case DG_ETIMEOUT: return "timed out";
    case DG_EMESH: return "invalid mesh";
    default: return "unknown status";
  }
}

const char* dg_last_error(const dg_ctx* ctx) {
  return ctx ? ctx->err.c_str() : g_setup_err.c_str();
}

int dg_mesh_setup_coef(const dg_mesh_desc* m, int k, int prec, double alpha, const double* rho,
                       const double* c, uintptr_t stream, dg_ctx** out);

int dg_mesh_setup(const dg_mesh_desc* m, int k, int prec, double alpha, uintptr_t stream,
                  dg_ctx** out) {
  return dg_mesh_setup_coef(m, k, prec, alpha, nullptr, nullptr, stream, out);
}

int dg_mesh_setup_coef(const dg_mesh_desc* m, int k, int prec, double alpha, const double* rho_h,
                       const double* c_h, uintptr_t stream, dg_ctx** out) {
  if (!out) return DG_EINVAL;
  *out = nullptr;
  g_setup_err.clear();
  if (!m || !m->nodes || !m->nbr || !m->nbr_face || !m->orient || m->n_elem < 1) {
    g_setup_err = "NULL mesh array or n_elem < 1";
    return DG_EINVAL;
  }
  if (k < 1 || k > DG_KMAX) {
    g_setup_err = "degree k outside [1, DG_KMAX]";
    return DG_EUNSUPPORTED;
  }
  if (m->geom_degree < 1 || m->geom_degree > DG_NMAX) {
    g_setup_err = "geometry degree outside [1, 8]";
    return DG_EUNSUPPORTED;
  }
  if (prec != DG_FP64 && prec != DG_FP32) {
    g_setup_err = "precision must be DG_FP64 or DG_FP32";
    return DG_EINVAL;
  }
  if (!(alpha >= 0.0 && alpha <= 1.0)) {
    g_setup_err = "flux_alpha outside [0, 1]";
    return DG_EINVAL;
  }
  int rc = validate_mesh(m, &g_setup_err);
  if (rc) return rc;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    g_setup_err = "no CUDA device";
    return DG_ECUDA;
  }
  if ((rc = init_device(dev, &g_setup_err))) return rc;

  dg_ctx* ctx = new (std::nothrow) dg_ctx();
  if (!ctx) return DG_ENOMEM;
  ctx->dev = dev;
  ctx->E = m->n_elem;
  ctx->Erun = m->n_elem;
  ctx->k = k;
  ctx->n = k + 1;
  ctx->q = m->geom_degree;
  ctx->prec = prec;
  ctx->alpha = alpha;
  ctx->rsize = prec == DG_FP64 ? 8 : 4;
  const int E = ctx->E, n = ctx->n, n3 = n * n * n, qc = ctx->q + 1;
  cudaStream_t st = S(stream);
  auto bail = [&](int code) {
    g_setup_err = ctx->err;
    delete ctx;
    return code;
  };
  ctx->tstride = tck_geo_stride(n, ctx->tstep);
  const size_t rs = ctx->rsize;
  if ((rc = ctx->alloc(&ctx->nbr, sizeof(int32_t) * 6 * E, "nbr")) ||
      (rc = ctx->alloc(&ctx->nbr_face, 6 * (size_t)E, "nbr_face")) ||
      (rc = ctx->alloc(&ctx->orient, 6 * (size_t)E, "orient")) ||
      (rc = ctx->alloc(&ctx->nodes, sizeof(double) * 3 * qc * qc * qc * (size_t)E, "nodes")) ||
      (rc = ctx->alloc(&ctx->rho, sizeof(double) * n3 * (size_t)E, "rho")) ||
      (rc = ctx->alloc(&ctx->c, sizeof(double) * n3 * (size_t)E, "c")) ||
      (rc = ctx->alloc(&ctx->pts, sizeof(double) * 3 * DG_PTS_LEN, "points")) ||
      (rc = ctx->alloc(&ctx->xq, sizeof(double) * (DG_NMAX + 2), "geometry points")) ||
      (rc = ctx->alloc(&ctx->bad, sizeof(int), "flag")) ||
      (rc = ctx->alloc(&ctx->geoA, rs * geo_stride_A(n) * (size_t)E, "cell metric")) ||
      (rc = ctx->alloc(&ctx->geoM, rs * geo_stride_M(n) * (size_t)E, "mass diagonal")) ||
      (rc = ctx->alloc(&ctx->geoF, rs * geo_stride_F(n) * (size_t)E, "face data")) ||
      (rc = ctx->alloc(&ctx->geoT, rs * (size_t)ctx->tstride * E, "predictor geometry")))
    return bail(rc);
  ctx->geo_affine = mesh_is_affine(m);
  if (ctx->geo_affine) {
    if ((rc = ctx->alloc(&ctx->geoK, rs * DG_AFF_OP * (size_t)E, "affine operator data")) ||
        (rc = ctx->alloc(&ctx->geoKT, rs * DG_AFF_TCK * (size_t)E, "affine predictor data")))
      return bail(rc);
    ctx->affine = coef_constant(rho_h, c_h, E, n3);
  }
  std::vector<double> hpts(3 * DG_PTS_LEN);
  std::memcpy(hpts.data(), g_tab.xg, sizeof(double) * DG_PTS_LEN);
  std::memcpy(hpts.data() + DG_PTS_LEN, g_tab.wg, sizeof(double) * DG_PTS_LEN);
  std::memcpy(hpts.data() + 2 * DG_PTS_LEN, g_tab.xgl, sizeof(double) * DG_PTS_LEN);
  std::vector<double> hxq(DG_NMAX + 2, 0.0);
  gauss_lobatto(qc, hxq.data());
  if ((rho_h == nullptr) != (c_h == nullptr)) {
    g_setup_err = "rho and c must both be given or both be NULL";
    delete ctx;
    return DG_EINVAL;
  }
  if (rho_h)
    for (size_t i = 0; i < (size_t)n3 * E; ++i)
      if (!(rho_h[i] > 0.0) || !(c_h[i] > 0.0) || !std::isfinite(rho_h[i]) || !std::isfinite(c_h[i])) {
        g_setup_err = "coefficients must be positive and finite";
        delete ctx;
        return DG_EINVAL;
      }
  std::vector<double> ones(rho_h ? 0 : (size_t)n3 * E, 1.0);
  const double* rho_src = rho_h ? rho_h : ones.data();
  const double* c_src = c_h ? c_h : ones.data();
  cudaError_t ce;
#define DG_UP(dst, src, bytes)                                                            \
  if ((ce = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st)) != cudaSuccess) { \
    ctx->cuda_fail(ce, "upload");                                                         \
    return bail(DG_ECUDA);                                                                \
  }
  DG_UP(ctx->nbr, m->nbr, sizeof(int32_t) * 6 * E);
  DG_UP(ctx->nbr_face, m->nbr_face, 6 * (size_t)E);
  DG_UP(ctx->orient, m->orient, 6 * (size_t)E);
  DG_UP(ctx->nodes, m->nodes, sizeof(double) * 3 * qc * qc * qc * (size_t)E);
  DG_UP(ctx->rho, rho_src, sizeof(double) * n3 * (size_t)E);
  DG_UP(ctx->c, c_src, sizeof(double) * n3 * (size_t)E);
  DG_UP(ctx->pts, hpts.data(), sizeof(double) * 3 * DG_PTS_LEN);
  DG_UP(ctx->xq, hxq.data(), sizeof(double) * (DG_NMAX + 2));
#undef DG_UP
  const int pi = ctx->prec;
  ctx->epb_op = pick_epb(n, g_kt.smem[pi][n](0, 2), 128, g_kt.maxthr[pi][n](0));
  ctx->epb_tck = pick_epb(n, g_kt.smem[pi][n](1, 2), 128, g_kt.maxthr[pi][n](1));
  ctx->epb_en = pick_epb(n, g_kt.smem[pi][n](2, 2), 128, g_kt.maxthr[pi][n](2));
  if ((rc = run_setup(ctx, st))) return bail(rc);
  *out = ctx;
  return DG_OK;
}

int dg_set_coefficients(dg_ctx* ctx, const double* rho, const double* c, uintptr_t stream) {
  if (!ctx) return DG_EINVAL;
  if (!rho || !c) return ctx->fail(DG_EINVAL, "NULL coefficient array");
  const size_t cnt = (size_t)ctx->E * ctx->npts();
  for (size_t i = 0; i < cnt; ++i)
    if (!(rho[i] > 0.0) || !(c[i] > 0.0) || !std::isfinite(rho[i]) || !std::isfinite(c[i]))
      return ctx->fail(DG_EINVAL, "coefficients must be positive and finite (index %zu)", i);
  DeviceGuard g(ctx->dev);
  cudaStream_t st = S(stream);
  DG_CK(cudaMemcpyAsync(ctx->rho, rho, sizeof(double) * cnt, cudaMemcpyHostToDevice, st), "upload rho");
  DG_CK(cudaMemcpyAsync(ctx->c, c, sizeof(double) * cnt, cudaMemcpyHostToDevice, st), "upload c");
  ctx->affine = ctx->dim == 3 && ctx->geo_affine && coef_constant(rho, c, ctx->E, ctx->npts());
  return run_setup(ctx, st);
}

int dg_apply_operator(dg_ctx* ctx, const void* U, void* R, uintptr_t stream) {
  if (!ctx) return DG_EINVAL;
  int rc;
  if ((rc = check_state_ptr(ctx, U, "U")) || (rc = check_state_ptr(ctx, R, "R"))) return rc;
  const char* u0 = static_cast<const char*>(U);
  const char* r0 = static_cast<const char*>(R);
  const size_t b = ctx->state_bytes();
  if (u0 < r0 + b && r0 < u0 + b) return ctx->fail(DG_EINVAL, "U and R overlap");
  DeviceGuard g(ctx->dev);
  if (ctx->dim == 2) return apply2(ctx, U, R, S(stream));
  OpParams p = op_params(ctx);
  p.U = U;
  p.out = R;
  return launch_op(ctx, p, EPI_WRITE, S(stream));
}

int dg_step_lsrk(dg_ctx* ctx, void* U, double dt, int32_t nsteps, uintptr_t stream) {
  if (!ctx) return DG_EINVAL;
  int rc;
  if ((rc = check_state_ptr(ctx, U, "U"))) return rc;
  if (!(dt > 0.0) || !std::isfinite(dt) || nsteps < 0)
    return ctx->fail(DG_EINVAL, "need dt > 0 and nsteps >= 0");
  DeviceGuard g(ctx->dev);
  return lsrk_steps(ctx, U, dt, nsteps, S(stream));
}

int dg_step_ader(dg_ctx* ctx, void* U, double dt, int32_t nsteps, int32_t red, uintptr_t stream) {
  if (!ctx) return DG_EINVAL;
  int rc;
  if ((rc = check_state_ptr(ctx, U, "U"))) return rc;
  if (!(dt > 0.0) || !std::isfinite(dt) || nsteps < 0)
    return ctx->fail(DG_EINVAL, "need dt > 0 and nsteps >= 0");
  if ((rc = check_red(ctx, red))) return rc;
  DeviceGuard g(ctx->dev);
  if ((rc = ensure_levels(ctx, red, S(stream)))) return rc;
  return ader_steps(ctx, U, dt, nsteps, red, S(stream));
}

int dg_step_hdg_ader(dg_ctx* ctx, void* U, double dt, int32_t nsteps, int32_t red, uintptr_t stream) {
  if (!ctx) return DG_EINVAL;
  int rc;
  if ((rc = check_state_ptr(ctx, U, "U"))) return rc;
  if (!(dt > 0.0) || !std::isfinite(dt) || nsteps < 0)
    return ctx->fail(DG_EINVAL, "need dt > 0 and nsteps >= 0");
  if ((rc = check_red(ctx, red))) return rc;
  DeviceGuard g(ctx->dev);
  if ((rc = ensure_levels(ctx, red, S(stream)))) return rc;
  return ader_steps(ctx, U, dt, nsteps, red, S(stream), true);
}

int dg_tck(dg_ctx* ctx, const void* U, void* Ubar, double dt, int32_t red, uintptr_t stream) {
  if (!ctx) return DG_EINVAL;
  int rc;
  if ((rc = check_state_ptr(ctx, U, "U")) || (rc = check_state_ptr(ctx, Ubar, "Ubar"))) return rc;
  if ((rc = check_red(ctx, red))) return rc;
  if (!std::isfinite(dt)) return ctx->fail(DG_EINVAL, "dt not finite");
  DeviceGuard g(ctx->dev);
  if (ctx->dim == 2) return tck2_gl(ctx, U, Ubar, dt, red, S(stream));
  if ((rc = ensure_levels(ctx, red, S(stream)))) return rc;
  return launch_tck(ctx, U, Ubar, dt, red, S(stream));
}

int dg_energy(dg_ctx* ctx, const void* U, double* out, uintptr_t stream) {
  if (!ctx || !out) return DG_EINVAL;
  int rc;
  if ((rc = check_state_ptr(ctx, U, "U"))) return rc;
  DeviceGuard g(ctx->dev);
  if (ctx->dim == 2) return energy2(ctx, U, out, S(stream));
  const int blocks = (ctx->Erun + ctx->epb_en - 1) / ctx->epb_en;
  if ((rc = ensure_partial(ctx, blocks))) return rc;
  EnergyParams p;
  p.U = U;
  p.geoM = ctx->geoM;
  p.partial = ctx->partial;
  p.E = ctx->Erun;
  cudaStream_t st = S(stream);
  DG_CK(g_kt.energy[ctx->prec][ctx->n](p, ctx->epb_en, st), "energy kernel launch");
  ctx->launches++;
  std::vector<double> h(blocks);
  DG_CK(cudaMemcpyAsync(h.data(), ctx->partial, sizeof(double) * blocks, cudaMemcpyDeviceToHost, st),
        "copy partials");
  DG_CK(cudaStreamSynchronize(st), "energy");
  double s = 0.0;
  for (int i = 0; i < blocks; ++i) s += h[i];
  *out = s;
  return DG_OK;
}

int dg_norms(dg_ctx* ctx, const void* A, const void* B, double* aa, double* dd, uintptr_t stream) {
  if (!ctx || !aa) return DG_EINVAL;
  int rc;
  if ((rc = check_state_ptr(ctx, A, "A"))) return rc;
  if (B && (rc = check_state_ptr(ctx, B, "B"))) return rc;
  DeviceGuard g(ctx->dev);
  const int blocks = 1024;
  if ((rc = ensure_partial(ctx, 2 * blocks))) return rc;
  cudaStream_t st = S(stream);
  const size_t cnt = ctx->run_elems();
  if (ctx->prec == DG_FP64)
    sumsq_kernel<double><<<blocks, 256, 0, st>>>(static_cast<const double*>(A),
                                                 static_cast<const double*>(B), cnt, ctx->partial);
  else
    sumsq_kernel<float><<<blocks, 256, 0, st>>>(static_cast<const float*>(A),
                                                static_cast<const float*>(B), cnt, ctx->partial);
  DG_CK(cudaGetLastError(), "norm kernel launch");
  ctx->launches++;
  std::vector<double> h(2 * blocks);
  DG_CK(cudaMemcpyAsync(h.data(), ctx->partial, sizeof(double) * 2 * blocks, cudaMemcpyDeviceToHost, st),
        "copy partials");
  DG_CK(cudaStreamSynchronize(st), "norms");
  double s1 = 0.0, s2 = 0.0;
  for (int i = 0; i < blocks; ++i) {
    s1 += h[2 * i];
    s2 += h[2 * i + 1];
  }
  *aa = s1;
  if (dd) *dd = s2;
  return DG_OK;
}

int dg_solve_host(dg_ctx* ctx, int method, const void* Uh, void* Uout, double dt, int32_t nsteps,
                  int32_t red, uintptr_t stream) {
  if (!ctx) return DG_EINVAL;
  if (!Uh || !Uout) return ctx->fail(DG_EINVAL, "NULL host buffer");
  if (method != 0 && method != 1) return ctx->fail(DG_EINVAL, "method must be 0 (LSRK) or 1 (ADER)");
  if (!(dt > 0.0) || nsteps < 0) return ctx->fail(DG_EINVAL, "need dt > 0 and nsteps >= 0");
  int rc;
  if (method == 1 && (rc = check_red(ctx, red))) return rc;
  DeviceGuard g(ctx->dev);
  if (method == 1 && (rc = ensure_levels(ctx, red, S(stream)))) return rc;
  if ((rc = ensure(ctx, &ctx->Uh, "host-solve state"))) return rc;
  cudaStream_t st = S(stream);
  const size_t b = ctx->state_bytes();
  // With Gauss-point states inside the steppers and host buffers the device
  // can address (pinned or managed memory), the transfers and the two changes
  // of basis are fused: one kernel reads the host state and writes its
  // Gauss-point values to the device, another writes the result back to the
  // host in the GL basis.  Otherwise: copies, and the steppers change basis.
  const void* din = ctx->dim == 3 ? device_view(Uh) : nullptr;
  void* dout = ctx->dim == 3 ? const_cast<void*>(device_view(Uout)) : nullptr;
  if (ctx->basis == DG_BASIS_G && nsteps > 0 && din && dout) {
    {
      dg_ctx::Span span(ctx, DG_KIND_OTHER, st);
      DG_CK(g_kt.basis[ctx->prec][ctx->n](din, ctx->Uh, ctx->Erun, 1, ctx->epb_en, st), "basis kernel launch");
      span.done();
      ctx->launches++;
    }
    rc = method == 0 ? lsrk_steps(ctx, ctx->Uh, dt, nsteps, st, true)
                     : ader_steps(ctx, ctx->Uh, dt, nsteps, red, st, false, true);
    if (rc) return rc;
    {
      dg_ctx::Span span(ctx, DG_KIND_OTHER, st);
      DG_CK(g_kt.basis[ctx->prec][ctx->n](ctx->Uh, dout, ctx->Erun, 0, ctx->epb_en, st), "basis kernel launch");
      span.done();
      ctx->launches++;
    }
  } else {
    DG_CK(cudaMemcpyAsync(ctx->Uh, Uh, b, cudaMemcpyHostToDevice, st), "copy in");
    rc = method == 0 ? lsrk_steps(ctx, ctx->Uh, dt, nsteps, st)
                     : ader_steps(ctx, ctx->Uh, dt, nsteps, red, st);
    if (rc) return rc;
    DG_CK(cudaMemcpyAsync(Uout, ctx->Uh, b, cudaMemcpyDeviceToHost, st), "copy out");
  }
  DG_CK(cudaStreamSynchronize(st), "solve");
  return dg_check_device(ctx, stream);
}

namespace {
// One FP64 <-> context-precision copy between a host array and a device
// state: to_host != 0 reads U into host, else writes host into U.
int state_copy(dg_ctx* ctx, void* U, double* host, int to_host, cudaStream_t st) {
  const size_t cnt = ctx->state_elems();
  if (ctx->prec == DG_FP64) {
    if (to_host)
      DG_CK(cudaMemcpyAsync(host, U, cnt * sizeof(double), cudaMemcpyDeviceToHost, st), "copy out");
    else
      DG_CK(cudaMemcpyAsync(U, host, cnt * sizeof(double), cudaMemcpyHostToDevice, st), "copy in");
    DG_CK(cudaStreamSynchronize(st), "state copy");
    return DG_OK;
  }
  void* tmp = nullptr;
  if (cudaMallocAsync(&tmp, cnt * sizeof(double), st) != cudaSuccess) {
    cudaGetLastError();
    return ctx->fail(DG_ENOMEM, "no room for a %zu-byte FP64 staging buffer", cnt * sizeof(double));
  }
  const int threads = 256;
  const int blocks = (int)std::min<size_t>((cnt + threads - 1) / threads, 4096);
  cudaError_t e = cudaSuccess;
  if (to_host) {
    cast_kernel<float, double><<<blocks, threads, 0, st>>>(static_cast<const float*>(U),
                                                          static_cast<double*>(tmp), cnt);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(host, tmp, cnt * sizeof(double), cudaMemcpyDeviceToHost, st);
  } else {
    e = cudaMemcpyAsync(tmp, host, cnt * sizeof(double), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
      cast_kernel<double, float><<<blocks, threads, 0, st>>>(static_cast<const double*>(tmp),
                                                            static_cast<float*>(U), cnt);
      e = cudaGetLastError();
    }
  }
  if (e == cudaSuccess) ctx->launches++;
  cudaError_t f = cudaFreeAsync(tmp, st);
  if (e == cudaSuccess) e = f;
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return ctx->cuda_fail(e, "state copy");
  return DG_OK;
}
}  // namespace

int dg_get_state(dg_ctx* ctx, const void* U, double* host_out, uintptr_t stream) {
  if (!ctx) return DG_EINVAL;
  if (!host_out) return ctx->fail(DG_EINVAL, "NULL host buffer");
  int rc;
  if ((rc = check_state_ptr(ctx, U, "U"))) return rc;
  DeviceGuard g(ctx->dev);
  return state_copy(ctx, const_cast<void*>(U), host_out, 1, S(stream));
}

int dg_set_state(dg_ctx* ctx, const double* host_in, void* U, uintptr_t stream) {
  if (!ctx) return DG_EINVAL;
  if (!host_in) return ctx->fail(DG_EINVAL, "NULL host buffer");
  int rc;
  if ((rc = check_state_ptr(ctx, U, "U"))) return rc;
  DeviceGuard g(ctx->dev);
  return state_copy(ctx, U, const_cast<double*>(host_in), 0, S(stream));
}

int dg_set_basis(dg_ctx* ctx, int basis) {
  if (!ctx) return DG_EINVAL;
  if (basis != DG_BASIS_GL && basis != DG_BASIS_G) return ctx->fail(DG_EINVAL, "basis must be DG_BASIS_GL or DG_BASIS_G");
  if (ctx->dim == 2 && basis != DG_BASIS_G)
    return ctx->fail(DG_EUNSUPPORTED, "2D meshes step in the Gauss basis only");
  ctx->basis = basis;
  return DG_OK;
}

int dg_get_basis(const dg_ctx* ctx) { return ctx ? ctx->basis : DG_EINVAL; }

int dg_set_predictor_kernel(dg_ctx* ctx, int kind) {
  if (!ctx) return DG_EINVAL;
  if (kind != DG_PRED_AUTO && kind != DG_PRED_LINES && kind != DG_PRED_COLUMNS && kind != DG_PRED_GL_PROJECTION &&
      kind != DG_PRED_INTERLEAVED)
    return ctx->fail(DG_EINVAL,
                     "predictor kernel must be DG_PRED_AUTO, DG_PRED_LINES, DG_PRED_COLUMNS, DG_PRED_GL_PROJECTION "
                     "or DG_PRED_INTERLEAVED");
  if (kind == DG_PRED_GL_PROJECTION && ctx->dim == 2)
    return ctx->fail(DG_EUNSUPPORTED, "not built for 2D meshes");
  ctx->pred_kernel = kind;
  return DG_OK;
}

int dg_get_predictor_kernel(const dg_ctx* ctx) { return ctx ? ctx->pred_kernel : DG_EINVAL; }

int dg_is_affine(const dg_ctx* ctx) { return ctx ? (ctx->affine ? 1 : 0) : DG_EINVAL; }

int dg_change_basis(dg_ctx* ctx, void* U, int to_g, uintptr_t stream) {
  if (!ctx) return DG_EINVAL;
  int rc;
  if ((rc = check_state_ptr(ctx, U, "U"))) return rc;
  DeviceGuard g(ctx->dev);
  return change_basis(ctx, U, to_g ? 1 : 0, S(stream));
}

int dg_check_device(dg_ctx* ctx, uintptr_t stream) {
  if (!ctx) return DG_EINVAL;
  DeviceGuard g(ctx->dev);
  cudaStream_t st = S(stream);
  int flag = 0;
  DG_CK(cudaMemcpyAsync(&flag, ctx->bad, sizeof(int), cudaMemcpyDeviceToHost, st), "read status");
  DG_CK(cudaStreamSynchronize(st), "status");
  if (flag) {
    DG_CK(cudaMemsetAsync(ctx->bad, 0, sizeof(int), st), "clear status");
    DG_CK(cudaStreamSynchronize(st), "status");
    return ctx->fail(DG_ETIMEOUT, "a bounded device wait gave up (its results were discarded)");
  }
  return DG_OK;
}

int dg_set_lsrk_scheme(dg_ctx* ctx, int32_t scheme) {
  if (!ctx) return DG_EINVAL;
  if (scheme != DG_LSRK_CK54 && scheme != DG_LSRK45 && scheme != DG_LSRK59)
    return ctx->fail(DG_EINVAL, "scheme must be DG_LSRK_CK54, DG_LSRK45 or DG_LSRK59 (got %d)", scheme);
  if (ctx->dim == 2 && scheme != DG_LSRK_CK54)
    return ctx->fail(DG_EUNSUPPORTED, "2D meshes step with DG_LSRK_CK54 only");
  ctx->lsrk_scheme = scheme;
  return DG_OK;
}

int dg_get_lsrk_scheme(const dg_ctx* ctx) { return ctx ? ctx->lsrk_scheme : DG_EINVAL; }

int dg_test_expire_waits(dg_ctx* ctx, int32_t on) {
  if (!ctx) return DG_EINVAL;
  ctx->expire_wait = on ? 1 : 0;
  return DG_OK;
}

int dg_info(const dg_ctx* ctx, int32_t* E, int32_t* k, int32_t* prec, size_t* bytes) {
  if (!ctx) return DG_EINVAL;
  if (E) *E = ctx->E;
  if (k) *k = ctx->k;
  if (prec) *prec = ctx->prec;
  if (bytes) *bytes = ctx->state_bytes();
  return DG_OK;
}

size_t dg_device_bytes(const dg_ctx* ctx) { return ctx ? ctx->dev_bytes : 0; }

int dg_profile_enable(dg_ctx* ctx, int enable) {
  if (!ctx) return DG_EINVAL;
  ctx->prof = enable != 0;
  return DG_OK;
}

int dg_profile_read(dg_ctx* ctx, double* ms, int64_t* launches, int reset) {
  if (!ctx || !ms || !launches) return DG_EINVAL;
  DeviceGuard g(ctx->dev);
  for (int i = 0; i < DG_NKINDS; ++i) {
    ms[i] = 0.0;
    launches[i] = 0;
  }
  for (auto& r : ctx->recs) {
    DG_CK(cudaEventSynchronize(r.b), "profile event");
    float t = 0.f;
    DG_CK(cudaEventElapsedTime(&t, r.a, r.b), "profile elapsed");
    ms[r.kind] += t;
    launches[r.kind] += 1;
  }
  if (reset) {
    for (auto& r : ctx->recs) {
      ctx->event_pool.push_back(r.a);
      ctx->event_pool.push_back(r.b);
    }
    ctx->recs.clear();
  }
  return DG_OK;
}

uint64_t dg_launch_count(const dg_ctx* ctx) { return ctx ? ctx->launches : 0; }

void dg_destroy(dg_ctx* ctx) { delete ctx; }

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free energy.  Same result as dg_energy, but the per-block
// partial sums live in a fixed device array that belongs to the library
// instead of context scratch allocated on first use, the final sum is done
// on the device, and the result goes to a caller-owned device double.  The
// call allocates no device memory and, when it succeeds, no host memory.
// ---------------------------------------------------------------------------
namespace {

// 16384 doubles = 128 KB, held by every GPU that loads the library until the
// process exits.  One slot per block of the energy kernel.
constexpr int kNoallocMaxPartials = 16384;
static __device__ __align__(256) double g_noalloc_partials[kNoallocMaxPartials];

constexpr int kNoallocMaxDevices = 64;
std::mutex g_noalloc_mu;
double* g_noalloc_addr[kNoallocMaxDevices] = {nullptr};  // device address of the array, per device

// Sum part[0..n) in a fixed order (strided per thread, then a fixed tree).
__global__ void noalloc_sum_kernel(const double* part, int n, double* out) {
  __shared__ double r[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += part[i];
  r[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) r[threadIdx.x] += r[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = r[0];
}

}  // namespace

extern "C" int dg_energy_noalloc(dg_ctx* ctx, const void* U, double* out, uintptr_t stream) {
  if (ctx && ctx->dim == 2) return ctx->fail(DG_EUNSUPPORTED, "not built for 2D meshes");
  if (!ctx) return DG_EINVAL;
  int rc;
  if ((rc = check_state_ptr(ctx, U, "U"))) return rc;
  if (!out) return ctx->fail(DG_EINVAL, "out is NULL");
  {  // the result is written by a kernel: out must be this device's memory
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, out) != cudaSuccess) {
      cudaGetLastError();
      return ctx->fail(DG_EINVAL, "out is not a device pointer");
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
      return ctx->fail(DG_EINVAL, "out must be device (or managed) memory, not host memory");
    if (a.type == cudaMemoryTypeDevice && a.device != ctx->dev)
      return ctx->fail(DG_EINVAL, "out is memory of device %d, the context is on device %d", a.device, ctx->dev);
    if (reinterpret_cast<uintptr_t>(out) % alignof(double) != 0)
      return ctx->fail(DG_EINVAL, "out must be 8-byte aligned");
  }
  if (ctx->dev < 0 || ctx->dev >= kNoallocMaxDevices)
    return ctx->fail(DG_EUNSUPPORTED, "dg_energy_noalloc serves devices 0..%d", kNoallocMaxDevices - 1);
  const int blocks = (ctx->Erun + ctx->epb_en - 1) / ctx->epb_en;
  if (blocks > kNoallocMaxPartials)
    return ctx->fail(DG_EINVAL,
                     "dg_energy_noalloc: this mesh needs %d partial sums but the fixed buffer "
                     "holds %d (at most %d elements at this degree and precision); use dg_energy",
                     blocks, kNoallocMaxPartials, kNoallocMaxPartials * ctx->epb_en);
  DeviceGuard g(ctx->dev);
  double* part = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[ctx->dev]) {
      // first call on this device: the host-side name of the array is only a
      // stand-in, so look up its device address with this device current
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
      if (e != cudaSuccess) {
        cudaGetLastError();
        return ctx->cuda_fail(e, "cudaGetSymbolAddress of the fixed partial-sum buffer");
      }
      g_noalloc_addr[ctx->dev] = static_cast<double*>(p);
    }
    part = g_noalloc_addr[ctx->dev];
  }
  // every slot the sum reads is written first by this call's energy kernel,
  // so nothing left over from an earlier call is used
  EnergyParams p;
  p.U = U;
  p.geoM = ctx->geoM;
  p.partial = part;
  p.E = ctx->Erun;
  cudaStream_t st = S(stream);
  DG_CK(g_kt.energy[ctx->prec][ctx->n](p, ctx->epb_en, st), "energy kernel launch");
  noalloc_sum_kernel<<<1, 256, 0, st>>>(part, blocks, out);
  DG_CK(cudaGetLastError(), "partial-sum kernel launch");
  ctx->launches += 2;
  return DG_OK;
}

// ---------------------------------------------------------------------------
// Tiling (elements per block) and its measurement, for the autotuner.
// ---------------------------------------------------------------------------
namespace {

int epb_ok(const dg_ctx* ctx, int which, int epb) {
  const int n = ctx->n;
  if (epb < 1 || epb * n * n > 1024 || epb * n * n > g_kt.maxthr[ctx->prec][n](which)) return 0;
  const int bytes = g_kt.smem[ctx->prec][n](which, 2);
  return (size_t)epb * bytes <= 200 * 1024;
}

}  // namespace

extern "C" int dg_set_tiling(dg_ctx* ctx, int32_t epb_op, int32_t epb_tck) {
  if (ctx && ctx->dim == 2) return ctx->fail(DG_EUNSUPPORTED, "not built for 2D meshes");
  if (!ctx) return DG_EINVAL;
  if (epb_op > 0) {
    if (!epb_ok(ctx, 0, epb_op)) return ctx->fail(DG_EINVAL, "elements per block %d not possible", epb_op);
    ctx->epb_op = epb_op;
  }
  if (epb_tck > 0) {
    if (!epb_ok(ctx, 1, epb_tck)) return ctx->fail(DG_EINVAL, "elements per block %d not possible", epb_tck);
    ctx->epb_tck = epb_tck;
  }
  return DG_OK;
}

extern "C" int dg_get_tiling(const dg_ctx* ctx, int32_t* epb_op, int32_t* epb_tck) {
  if (!ctx) return DG_EINVAL;
  if (epb_op) *epb_op = ctx->epb_op;
  if (epb_tck) *epb_tck = ctx->epb_tck;
  return DG_OK;
}

extern "C" int dg_tune(dg_ctx* ctx, int kind, const int32_t* cand, int32_t ncand, int32_t reps,
                       double* ms_out, uintptr_t stream) {
  if (ctx && ctx->dim == 2) return ctx->fail(DG_EUNSUPPORTED, "not built for 2D meshes");
  if (!ctx || !cand || !ms_out || ncand < 1 || reps < 1) return DG_EINVAL;
  if (kind != DG_KIND_LSRK && kind != DG_KIND_TCK && kind != DG_KIND_ADER)
    return ctx->fail(DG_EINVAL, "kind must be DG_KIND_LSRK, DG_KIND_ADER or DG_KIND_TCK");
  DeviceGuard g(ctx->dev);
  int rc;
  if ((rc = ensure(ctx, &ctx->U2, "tuning state")) || (rc = ensure(ctx, &ctx->U3, "tuning state")) ||
      (rc = ensure(ctx, &ctx->dU, "tuning register")) || (rc = ensure(ctx, &ctx->Ubar, "tuning state")))
    return rc;
  cudaStream_t st = S(stream);
  DG_CK(cudaMemsetAsync(ctx->U2, 0, ctx->state_bytes(), st), "memset");
  DG_CK(cudaMemsetAsync(ctx->dU, 0, ctx->state_bytes(), st), "memset");
  const int which = kind == DG_KIND_TCK ? 1 : 0;
  const int saved = which ? ctx->epb_tck : ctx->epb_op;
  cudaEvent_t a = nullptr, b = nullptr;
  DG_CK(cudaEventCreate(&a), "event");
  DG_CK(cudaEventCreate(&b), "event");
  double best = 1e300;
  int best_epb = saved;
  for (int c = 0; c < ncand; ++c) {
    ms_out[c] = -1.0;
    if (!epb_ok(ctx, which, cand[c])) continue;
    if (which) ctx->epb_tck = cand[c]; else ctx->epb_op = cand[c];
    OpParams p = op_params(ctx);
    p.U = ctx->U2;
    p.Uadd = ctx->U2;
    p.out = ctx->U3;
    p.dU = ctx->dU;
    p.cA = 0.5;
    p.cB = 0.5;
    p.dt = 1e-3;
    for (int r = -1; r < reps; ++r) {  // one untimed launch first
      if (r == 0) cudaEventRecord(a, st);
      const bool gb = ctx->basis == DG_BASIS_G;  // time the kernels the steppers use
      if (kind == DG_KIND_TCK)
        rc = launch_tck(ctx, ctx->U2, ctx->Ubar, 1e-3, 2, st, gb);
      else
        rc = launch_op(ctx, p, kind == DG_KIND_LSRK ? EPI_LSRK : EPI_ADD, st, gb);
      if (rc) break;
    }
    if (rc) {  // launch configuration refused: not a candidate
      cudaGetLastError();
      rc = DG_OK;
      cudaStreamSynchronize(st);
      continue;
    }
    cudaEventRecord(b, st);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    ms_out[c] = ms / reps;
    if (ms_out[c] < best) {
      best = ms_out[c];
      best_epb = cand[c];
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (which) ctx->epb_tck = best_epb; else ctx->epb_op = best_epb;
  return rc;
}

// ---------------------------------------------------------------------------
// Batched form: independent solves advanced together by persistent launches.
// ---------------------------------------------------------------------------
// Solves of one degree in a batch: their work items and launch shape.
struct BatchGroup {
  int n = 0;
  int aff = 0;  // affine elements with constant coefficients (compact kernels in the Gauss basis)
  BatchItem* items_op = nullptr;
  BatchItem* items_tck = nullptr;
  BatchItem* slices_tckc = nullptr;  // FP32 column-form predictor: one block per slice
  int n_op = 0, n_tck = 0, n_tckc = 0;
  int block_op = 0, block_tck = 0, grid_op = 0, grid_tck[3] = {0, 0, 0};
  size_t smem_op = 0, smem_tck[3] = {0, 0, 0}, smem_tckc[3] = {0, 0, 0};  // [1] reduction 2, [2] none
  cudaStream_t s = nullptr;  // branch stream
  cudaEvent_t done = nullptr;
};

struct dg_batch {
  int dev = 0, prec = 0, n = 0;
  std::vector<dg_ctx*> ctx;
  std::vector<BatchGroup> groups;
  std::vector<void*> allocs;
  BatchInst* inst = nullptr;
  std::vector<BatchInst> hinst;  // host copy (re-uploaded when the basis changes)
  int* counters = nullptr;  // kCounters + 2 per group
  int basis = DG_BASIS_GL;
  bool convert_each_call = true;
  cudaEvent_t fork = nullptr;
  cudaStream_t cap = nullptr;  // private stream used for graph capture
  cudaGraphExec_t gexec[3] = {nullptr, nullptr, nullptr};  // ADER red 0, ADER red 2, LSRK
  uint64_t launches = 0;
  size_t dev_bytes = 0;
  std::string err;
  static constexpr int kChunk = 8;  // steps per captured graph
  static constexpr int kCounters = 5 * kChunk;
  static constexpr int kSlots = kCounters + 2;  // + the two changes of basis

  int fail(int code, const char* msg) {
    err = msg;
    return code;
  }
  ~dg_batch() {
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(dev);
    for (auto& g : gexec)
      if (g) cudaGraphExecDestroy(g);
    for (auto& g : groups) {
      if (g.s) cudaStreamDestroy(g.s);
      if (g.done) cudaEventDestroy(g.done);
    }
    if (fork) cudaEventDestroy(fork);
    if (cap) cudaStreamDestroy(cap);
    for (void* p : allocs) cudaFree(p);
    cudaSetDevice(cur);
  }
};

namespace {

int batch_alloc(dg_batch* b, void** p, size_t bytes) {
  if (cudaMalloc(p, bytes ? bytes : 16) != cudaSuccess) {
    cudaGetLastError();
    return b->fail(DG_ENOMEM, "cudaMalloc for batch tables failed");
  }
  b->allocs.push_back(*p);
  b->dev_bytes += bytes;
  return DG_OK;
}

// `steps` steps of one method: the degree groups branch off `st`, each runs
// its phases on its own stream, and `st` waits for all of them.
int batch_launch_steps(dg_batch* b, int method, int red, int steps, cudaStream_t st) {
  const int ng = (int)b->groups.size();
  cudaError_t e = cudaMemsetAsync(b->counters, 0, sizeof(int) * dg_batch::kSlots * ng, st);
  if (e == cudaSuccess) e = cudaEventRecord(b->fork, st);
  if (e != cudaSuccess) return b->fail(DG_ECUDA, cudaGetErrorString(e));
  const int ti = red == 2 ? 1 : 2;
  auto op = b->prec == DG_FP64 ? launch_batch_op_f64 : launch_batch_op_f32;
  auto tck = b->prec == DG_FP64 ? launch_batch_tck_f64 : launch_batch_tck_f32;
  for (int gi = 0; gi < ng && e == cudaSuccess; ++gi) {
    BatchGroup& g = b->groups[gi];
    int* cnt = b->counters + gi * dg_batch::kSlots;
    const int mode = b->basis == DG_BASIS_G ? (g.aff ? 2 : 1) : 0;
    e = cudaStreamWaitEvent(g.s, b->fork, 0);
    for (int s = 0; s < steps && e == cudaSuccess; ++s) {
      if (method == 1) {  // ADER: predictor, then update (FP32 Gauss-point states: column form)
        const bool col = b->prec == DG_FP32 && b->basis == DG_BASIS_G;
        if (col)
          e = tck(g.n, g.slices_tckc, g.n_tckc, b->inst, red, cnt++, 0, g.block_tck, g.smem_tckc[ti], g.s,
                  g.aff ? 2 : 1);
        else
          e = tck(g.n, g.items_tck, g.n_tck, b->inst, red, cnt++, g.grid_tck[ti], g.block_tck, g.smem_tck[ti], g.s, 0);
        if (e == cudaSuccess)
          e = op(g.n, g.items_op, g.n_op, b->inst, 5, cnt++, g.grid_op, g.block_op, g.smem_op, g.s, mode);
        b->launches += 2;
      } else {
        for (int ph = 0; ph < 5 && e == cudaSuccess; ++ph) {
          e = op(g.n, g.items_op, g.n_op, b->inst, ph, cnt++, g.grid_op, g.block_op, g.smem_op, g.s, mode);
          b->launches += 1;
        }
      }
    }
    if (e == cudaSuccess) e = cudaEventRecord(g.done, g.s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, g.done, 0);
  }
  if (e != cudaSuccess) return b->fail(DG_ECUDA, cudaGetErrorString(e));
  return DG_OK;
}

// In-place change of basis of every solve's state (GL -> G if to_g).
int batch_convert(dg_batch* b, int to_g, cudaStream_t st) {
  const int ng = (int)b->groups.size();
  auto conv = b->prec == DG_FP64 ? launch_batch_basis_f64 : launch_batch_basis_f32;
  cudaError_t e = cudaSuccess;
  for (int gi = 0; gi < ng && e == cudaSuccess; ++gi)
    e = cudaMemsetAsync(b->counters + gi * dg_batch::kSlots + dg_batch::kCounters + to_g, 0, sizeof(int), st);
  if (e == cudaSuccess) e = cudaEventRecord(b->fork, st);
  for (int gi = 0; gi < ng && e == cudaSuccess; ++gi) {
    BatchGroup& g = b->groups[gi];
    e = cudaStreamWaitEvent(g.s, b->fork, 0);
    if (e == cudaSuccess)
      e = conv(g.n, g.items_op, g.n_op, b->inst, to_g, b->counters + gi * dg_batch::kSlots + dg_batch::kCounters + to_g,
               g.grid_op, g.block_op, g.smem_op, g.s);
    b->launches += 1;
    if (e == cudaSuccess) e = cudaEventRecord(g.done, g.s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, g.done, 0);
  }
  if (e != cudaSuccess) return b->fail(DG_ECUDA, cudaGetErrorString(e));
  return DG_OK;
}

}  // namespace

extern "C" int dg_batch_create(dg_ctx* const* ctxs, void* const* U, const double* dt, int32_t n,
                               uintptr_t stream, dg_batch** out) {
  if (!out) return DG_EINVAL;
  *out = nullptr;
  g_setup_err.clear();
  if (!ctxs || !U || !dt || n < 1) {
    g_setup_err = "dg_batch_create: NULL arrays or n < 1";
    return DG_EINVAL;
  }
  const int prec = ctxs[0] ? ctxs[0]->prec : 0, dev = ctxs[0] ? ctxs[0]->dev : 0;
  for (int i = 0; i < n; ++i) {
    if (ctxs[i] && ctxs[i]->dim == 2) {
      g_setup_err = "batches are not built for 2D meshes";
      return DG_EUNSUPPORTED;
    }
    if (!ctxs[i] || ctxs[i]->prec != prec || ctxs[i]->dev != dev) {
      g_setup_err = "dg_batch_create: contexts must be non-NULL, of one precision and one device";
      return DG_EINVAL;
    }
    if (!(dt[i] > 0.0)) {
      g_setup_err = "dg_batch_create: dt must be positive";
      return DG_EINVAL;
    }
    if (check_state_ptr(ctxs[i], U[i], "U")) {
      g_setup_err = ctxs[i]->err;
      return DG_EINVAL;
    }
  }
  DeviceGuard dg_(dev);
  dg_batch* b = new (std::nothrow) dg_batch();
  if (!b) return DG_ENOMEM;
  b->dev = dev;
  b->prec = prec;
  b->n = n;
  auto bail = [&](int code) {
    g_setup_err = b->err;
    delete b;
    return code;
  };
  std::vector<BatchInst> hinst(n);
  // groups: index 2 n + aff
  std::vector<std::vector<BatchItem>> hop(2 * (DG_NMAX + 1)), htck(2 * (DG_NMAX + 1));
  auto maxthr = prec == DG_FP64 ? batch_max_threads_f64 : batch_max_threads_f32;
  std::vector<BatchGroup> byn(2 * (DG_NMAX + 1));
  for (int i = 0; i < n; ++i) {
    dg_ctx* c = ctxs[i];
    int rc;
    if ((rc = ensure(c, &c->U2, "LSRK state")) || (rc = ensure(c, &c->U3, "LSRK state")) ||
        (rc = ensure(c, &c->dU, "LSRK register")) || (rc = ensure(c, &c->Ubar, "ADER predictor"))) {
      b->err = c->err;
      return bail(rc);
    }
    BatchInst& I = hinst[i];
    std::memset(&I, 0, sizeof(I));
    void* const chain[6] = {U[i], c->U2, c->U3, c->U2, c->U3, U[i]};
    for (int s = 0; s < 5; ++s) {
      I.op[s] = op_params(c);
      I.op[s].U = chain[s];
      I.op[s].Uadd = chain[s];
      I.op[s].out = chain[s + 1];
      I.op[s].dU = c->dU;
      I.op[s].cA = kLsrkA[s];
      I.op[s].cB = kLsrkB[s];
      I.op[s].dt = dt[i];
      I.op[s].first = s == 0;
    }
    I.op[5] = op_params(c);
    I.op[5].U = c->Ubar;
    I.op[5].Uadd = U[i];
    I.op[5].out = U[i];
    I.tck.U = U[i];
    I.tck.Ubar = c->Ubar;
    I.tck.geoT = c->geoT;
    I.tck.geoT_stride = c->tstride;
    I.tck.geo_step = c->tstep;
    I.tck.E = c->Erun;
    I.tck.aff = c->affine ? 1 : 0;
    I.tck.geoKT = c->geoKT;
    double fact = 1.0;
    for (int j = 0; j <= c->n; ++j) {
      fact *= (j + 1);
      I.tck.coef[j] = std::pow(dt[i], j + 1) / fact;
    }
    const int nn = c->n, n2 = nn * nn, gk = 2 * nn + (c->affine ? 1 : 0);
    const int eo = std::max(1, std::min(c->epb_op, maxthr(nn, 0) / n2));
    const int et = std::max(1, std::min(c->epb_tck, maxthr(nn, 1) / n2));
    // items are cut below, once each group's launch shape is known
    hop[gk].push_back({i, 0, c->Erun, nn, eo});
    htck[gk].push_back({i, 0, c->Erun, nn, et});
    BatchGroup& g = byn[gk];
    g.n = nn;
    g.aff = c->affine ? 1 : 0;
    g.block_op = std::max(g.block_op, eo * n2);
    g.block_tck = std::max(g.block_tck, et * n2);
    g.smem_op = std::max(g.smem_op, (size_t)eo * g_kt.smem[prec][nn](0, 2));
    g.smem_tck[1] = std::max(g.smem_tck[1], (size_t)et * g_kt.smem[prec][nn](1, 2));
    g.smem_tck[2] = std::max(g.smem_tck[2], (size_t)et * g_kt.smem[prec][nn](1, 0));
    if (prec == DG_FP32) {
      g.smem_tckc[1] = std::max(g.smem_tckc[1], (size_t)et * g_kt.tckc_smem[prec][nn](2));
      g.smem_tckc[2] = std::max(g.smem_tckc[2], (size_t)et * g_kt.tckc_smem[prec][nn](0));
    }
    b->ctx.push_back(c);
  }
  // Item order: largest solves first (balance at the end of a launch), and
  // within a solve in element order, so that the blocks in flight sweep a
  // contiguous range of one solve and neighbours' face values are still in L2.
  std::vector<int> ecount(n);
  for (int i = 0; i < n; ++i) ecount[i] = ctxs[i]->E;
  auto by_size = [&](const BatchItem& x, const BatchItem& y) {
    if (x.inst != y.inst) return ecount[x.inst] != ecount[y.inst] ? ecount[x.inst] > ecount[y.inst] : x.inst < y.inst;
    return x.e0 < y.e0;
  };
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  auto occ = prec == DG_FP64 ? batch_occupancy_f64 : batch_occupancy_f32;
  int rc;
  if ((rc = batch_alloc(b, (void**)&b->inst, sizeof(BatchInst) * n))) return bail(rc);
  cudaStream_t st = S(stream);
  cudaError_t e = cudaMemcpyAsync(b->inst, hinst.data(), sizeof(BatchInst) * n, cudaMemcpyHostToDevice, st);
  for (int gk = 4; gk < 2 * (DG_NMAX + 1) && e == cudaSuccess; ++gk) {
    if (hop[gk].empty()) continue;
    const int nn = gk / 2;
    BatchGroup g = byn[gk];
    g.grid_op = sms * std::max(1, occ(nn, 0, g.block_op, g.smem_op));
    g.grid_tck[1] = sms * std::max(1, occ(nn, 1, g.block_tck, g.smem_tck[1]));
    g.grid_tck[2] = sms * std::max(1, occ(nn, 2, g.block_tck, g.smem_tck[2]));
    // the column form's slices: every solve in blocks of its own elements per
    // block, in the order of the work items (largest solves first)
    std::vector<BatchItem> slices;
    if (prec == DG_FP32) {
      std::vector<BatchItem> whole = htck[gk];
      std::sort(whole.begin(), whole.end(), by_size);
      for (const auto& w : whole)
        for (int e0 = w.e0; e0 < w.e0 + w.ne; e0 += w.epb)
          slices.push_back({w.inst, e0, std::min(w.epb, w.e0 + w.ne - e0), w.n, w.epb});
    }
    // cut each solve into items of about (elements of the degree) / (8 x
    // blocks) elements, in whole slices, so every block sees ~8 items
    auto cut = [](std::vector<BatchItem>& v, int grid) {
      long long tot = 0;
      for (const auto& w : v) tot += w.ne;
      std::vector<BatchItem> out;
      for (const auto& w : v) {
        long long per = std::max<long long>(w.epb, tot / (8LL * grid));
        per = (per + w.epb - 1) / w.epb * w.epb;
        for (int e0 = 0; e0 < w.ne; e0 += (int)per)
          out.push_back({w.inst, e0, (int)std::min<long long>(per, w.ne - e0), w.n, w.epb});
      }
      v.swap(out);
    };
    cut(hop[gk], g.grid_op);
    cut(htck[gk], std::max(g.grid_tck[1], g.grid_tck[2]));
    std::sort(hop[gk].begin(), hop[gk].end(), by_size);
    std::sort(htck[gk].begin(), htck[gk].end(), by_size);
    g.n_op = (int)hop[gk].size();
    g.n_tck = (int)htck[gk].size();
    g.n_tckc = (int)slices.size();
    if ((rc = batch_alloc(b, (void**)&g.items_op, sizeof(BatchItem) * g.n_op)) ||
        (rc = batch_alloc(b, (void**)&g.items_tck, sizeof(BatchItem) * g.n_tck)))
      return bail(rc);
    if (g.n_tckc && (rc = batch_alloc(b, (void**)&g.slices_tckc, sizeof(BatchItem) * g.n_tckc))) return bail(rc);
    e = cudaMemcpyAsync(g.items_op, hop[gk].data(), sizeof(BatchItem) * g.n_op, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(g.items_tck, htck[gk].data(), sizeof(BatchItem) * g.n_tck, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && g.n_tckc) {
      e = cudaMemcpyAsync(g.slices_tckc, slices.data(), sizeof(BatchItem) * g.n_tckc, cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // slices goes out of scope with this iteration
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&g.s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g.done, cudaEventDisableTiming);
    b->groups.push_back(g);
  }
  if (e == cudaSuccess)
    if ((rc = batch_alloc(b, (void**)&b->counters, sizeof(int) * dg_batch::kSlots * b->groups.size())))
      return bail(rc);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    b->fail(DG_ECUDA, cudaGetErrorString(e));
    return bail(DG_ECUDA);
  }
  b->hinst = std::move(hinst);
  *out = b;
  return DG_OK;
}

static int batch_steps(dg_batch* b, int method, int red, int32_t nsteps, uintptr_t stream) {
  DeviceGuard g(b->dev);
  cudaStream_t st = S(stream);
  const int gi = method == 0 ? 2 : (red == 2 ? 1 : 0);
  const int chunks = nsteps / dg_batch::kChunk, rest = nsteps % dg_batch::kChunk;
  const uint64_t per_chunk = (uint64_t)dg_batch::kChunk * (method == 0 ? 5 : 2) * b->groups.size();
  const bool conv = b->basis == DG_BASIS_G && b->convert_each_call && nsteps > 0;
  if (conv) {
    const int rc = batch_convert(b, 1, st);
    if (rc) return rc;
  }
  if (chunks > 0 && !b->gexec[gi]) {
    // capture kChunk steps once; the graph is replayed on the caller's stream
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return b->fail(DG_ECUDA, cudaGetErrorString(e));
    const uint64_t l0 = b->launches;
    int rc = batch_launch_steps(b, method, red, dg_batch::kChunk, b->cap);
    b->launches = l0;
    e = cudaStreamEndCapture(b->cap, &graph);
    if (rc) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    if (e != cudaSuccess) return b->fail(DG_ECUDA, cudaGetErrorString(e));
    e = cudaGraphInstantiate(&b->gexec[gi], graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      b->gexec[gi] = nullptr;
      return b->fail(DG_ECUDA, cudaGetErrorString(e));
    }
  }
  for (int c = 0; c < chunks; ++c) {
    cudaError_t e = cudaGraphLaunch(b->gexec[gi], st);
    if (e != cudaSuccess) return b->fail(DG_ECUDA, cudaGetErrorString(e));
    b->launches += per_chunk;
  }
  if (rest) {
    const int rc = batch_launch_steps(b, method, red, rest, st);
    if (rc) return rc;
  }
  if (conv) return batch_convert(b, 0, st);
  return DG_OK;
}

extern "C" int dg_batch_set_basis(dg_batch* b, int basis, int convert_each_call) {
  if (!b) return DG_EINVAL;
  if (basis != DG_BASIS_GL && basis != DG_BASIS_G) return b->fail(DG_EINVAL, "basis must be DG_BASIS_GL or DG_BASIS_G");
  DeviceGuard g(b->dev);
  b->basis = basis;
  b->convert_each_call = convert_each_call != 0;
  for (auto& I : b->hinst) I.tck.gmode = basis == DG_BASIS_G ? 1 : 0;
  cudaError_t e = cudaMemcpy(b->inst, b->hinst.data(), sizeof(BatchInst) * b->hinst.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return b->fail(DG_ECUDA, cudaGetErrorString(e));
  for (auto& x : b->gexec)  // captured graphs refer to the old kernels
    if (x) {
      cudaGraphExecDestroy(x);
      x = nullptr;
    }
  return DG_OK;
}

extern "C" int dg_batch_convert(dg_batch* b, int to_g, uintptr_t stream) {
  if (!b) return DG_EINVAL;
  DeviceGuard g(b->dev);
  return batch_convert(b, to_g ? 1 : 0, S(stream));
}

extern "C" int dg_batch_step_ader(dg_batch* b, int32_t nsteps, int32_t red, uintptr_t stream) {
  if (!b || nsteps < 0) return DG_EINVAL;
  if (red != 0 && red != 2)
    return b->fail(DG_EUNSUPPORTED, "batches take reduce_every 0 or 2 (1 and 3: dg_step_ader per solve)");
  return batch_steps(b, 1, red, nsteps, stream);
}

extern "C" int dg_batch_step_lsrk(dg_batch* b, int32_t nsteps, uintptr_t stream) {
  if (!b || nsteps < 0) return DG_EINVAL;
  for (dg_ctx* c : b->ctx)
    if (c->lsrk_scheme != DG_LSRK_CK54)
      return b->fail(DG_EUNSUPPORTED, "batches step LSRK with DG_LSRK_CK54 only");
  return batch_steps(b, 0, 0, nsteps, stream);
}

extern "C" int dg_batch_info(const dg_batch* b, int32_t* n_inst, int32_t* n_items, int32_t* block,
                             int32_t* grid, uint64_t* launches) {
  if (!b) return DG_EINVAL;
  int items = 0, blk = 0, grd = 0;
  for (const auto& g : b->groups) {
    items += g.n_op;
    blk = std::max(blk, g.block_op);
    grd += g.grid_op;
  }
  if (n_inst) *n_inst = b->n;
  if (n_items) *n_items = items;
  if (block) *block = blk;
  if (grid) *grid = grd;
  if (launches) *launches = b->launches;
  return DG_OK;
}

extern "C" const char* dg_batch_last_error(const dg_batch* b) { return b ? b->err.c_str() : ""; }

extern "C" void dg_batch_destroy(dg_batch* b) { delete b; }

// ---------------------------------------------------------------------------
// Partitioned solve: one mesh split into parts, each a context whose first
// n_owned elements are stepped and whose remaining elements are ghost copies
// of neighbours owned by other parts.  Before every operator application the
// ghost tiles of its input are refreshed from their owners (five exchanges
// per LSRK step, one per ADER step: the predictor is element-local, Sec. 4.1, 4.8).
// All parts live on this device; the exchange is one gather kernel.
// ---------------------------------------------------------------------------
extern "C" int dg_set_owned(dg_ctx* ctx, int32_t n_owned) {
  if (!ctx) return DG_EINVAL;
  if (ctx->dim == 2) return ctx->fail(DG_EUNSUPPORTED, "not built for 2D meshes");
  if (n_owned < 1 || n_owned > ctx->E)
    return ctx->fail(DG_EINVAL, "n_owned %d outside [1, %d]", n_owned, ctx->E);
  ctx->Erun = n_owned;
  return DG_OK;
}

namespace {

constexpr int DG_PART_MAX = 64;
struct PartPtrs {
  void* p[DG_PART_MAX];
};

// Block g copies ghost tile g: dst part / element <- src part / element,
// `words` 16-byte words per tile.
__global__ void ghost_copy_kernel(PartPtrs bufs, const int32_t* __restrict__ map, int words) {
  const int g = blockIdx.x;
  const int dp = map[4 * g], de = map[4 * g + 1], sp = map[4 * g + 2], se = map[4 * g + 3];
  const int4* src = static_cast<const int4*>(bufs.p[sp]) + (size_t)se * words;
  int4* dst = static_cast<int4*>(bufs.p[dp]) + (size_t)de * words;
  for (int i = threadIdx.x; i < words; i += blockDim.x) dst[i] = src[i];
}

}  // namespace

struct dg_part {
  int dev = 0, P = 0, nghost = 0, words = 0;
  std::vector<dg_ctx*> c;
  std::vector<void*> U;
  int32_t* map = nullptr;  // [nghost][4]: dst part, dst element, src part, src element
  uint64_t launches = 0;
  std::string err;
  int fail(int code, const char* msg) {
    err = msg;
    return code;
  }
  ~dg_part() {
    if (map) {
      int cur = 0;
      cudaGetDevice(&cur);
      cudaSetDevice(dev);
      cudaFree(map);
      cudaSetDevice(cur);
    }
  }
};

namespace {

int part_exchange(dg_part* t, void* const* bufs, cudaStream_t st) {
  if (!t->nghost) return DG_OK;
  PartPtrs pp;
  std::memset(&pp, 0, sizeof(pp));
  for (int i = 0; i < t->P; ++i) pp.p[i] = bufs[i];
  ghost_copy_kernel<<<t->nghost, 128, 0, st>>>(pp, t->map, t->words);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return t->fail(DG_ECUDA, cudaGetErrorString(e));
  t->launches++;
  return DG_OK;
}

int part_lsrk(dg_part* t, double dt, int nsteps, cudaStream_t st) {
  int rc;
  const int P = t->P;
  for (int i = 0; i < P; ++i)
    if (t->c[i]->lsrk_scheme != DG_LSRK_CK54)
      return t->fail(DG_EUNSUPPORTED, "partitioned solves step LSRK with DG_LSRK_CK54 only");
  for (int i = 0; i < P; ++i) {
    dg_ctx* c = t->c[i];
    if ((rc = ensure(c, &c->U2, "LSRK state")) || (rc = ensure(c, &c->U3, "LSRK state")) ||
        (rc = ensure(c, &c->dU, "LSRK register")))
      return t->fail(rc, c->err.c_str());
  }
  const bool g = t->c[0]->basis == DG_BASIS_G && nsteps > 0;
  if (g)
    for (int i = 0; i < P; ++i)
      if ((rc = change_basis(t->c[i], t->U[i], 1, st))) return t->fail(rc, t->c[i]->err.c_str());
  std::vector<void*> in(P);
  for (int s = 0; s < nsteps; ++s)
    for (int st5 = 0; st5 < 5; ++st5) {
      for (int i = 0; i < P; ++i) {
        dg_ctx* c = t->c[i];
        void* const chain[6] = {t->U[i], c->U2, c->U3, c->U2, c->U3, t->U[i]};
        in[i] = chain[st5];
      }
      if ((rc = part_exchange(t, in.data(), st))) return rc;
      for (int i = 0; i < P; ++i) {
        dg_ctx* c = t->c[i];
        void* const chain[6] = {t->U[i], c->U2, c->U3, c->U2, c->U3, t->U[i]};
        OpParams p = op_params(c);
        p.U = chain[st5];
        p.Uadd = chain[st5];
        p.out = chain[st5 + 1];
        p.dU = c->dU;
        p.cA = kLsrkA[st5];
        p.cB = kLsrkB[st5];
        p.dt = dt;
        p.first = st5 == 0;
        if ((rc = launch_op(c, p, EPI_LSRK, st, g))) return t->fail(rc, c->err.c_str());
      }
    }
  if (g)
    for (int i = 0; i < P; ++i)
      if ((rc = change_basis(t->c[i], t->U[i], 0, st))) return t->fail(rc, t->c[i]->err.c_str());
  return DG_OK;
}

int part_ader(dg_part* t, double dt, int nsteps, int red, cudaStream_t st, bool hdg = false) {
  int rc;
  const int P = t->P;
  for (int i = 0; i < P; ++i) {
    dg_ctx* c = t->c[i];
    if ((rc = ensure(c, &c->Ubar, "ADER predictor")) || (rc = ensure_levels(c, red, st)) ||
        (hdg && (rc = ensure(c, &c->Wd, "HDG-ADER derivative"))))
      return t->fail(rc, c->err.c_str());
  }
  const bool g = t->c[0]->basis == DG_BASIS_G && nsteps > 0;
  if (g)
    for (int i = 0; i < P; ++i)
      if ((rc = change_basis(t->c[i], t->U[i], 1, st))) return t->fail(rc, t->c[i]->err.c_str());
  std::vector<void*> bar(P);
  for (int i = 0; i < P; ++i) bar[i] = t->c[i]->Ubar;
  for (int s = 0; s < nsteps; ++s) {
    if (hdg) {  // the DG derivative needs the state's ghosts
      if ((rc = part_exchange(t, t->U.data(), st))) return rc;
      for (int i = 0; i < P; ++i) {
        dg_ctx* c = t->c[i];
        OpParams q = op_params(c);
        q.U = t->U[i];
        q.out = c->Wd;
        if ((rc = launch_op(c, q, EPI_WRITE, st, g))) return t->fail(rc, c->err.c_str());
      }
    }
    for (int i = 0; i < P; ++i)
      if ((rc = launch_tck(t->c[i], t->U[i], t->c[i]->Ubar, dt, red, st, g, hdg ? t->c[i]->Wd : nullptr)))
        return t->fail(rc, t->c[i]->err.c_str());
    if ((rc = part_exchange(t, bar.data(), st))) return rc;
    for (int i = 0; i < P; ++i) {
      dg_ctx* c = t->c[i];
      OpParams p = op_params(c);
      p.U = c->Ubar;
      p.Uadd = t->U[i];
      p.out = t->U[i];
      if ((rc = launch_op(c, p, EPI_ADD, st, g))) return t->fail(rc, c->err.c_str());
    }
  }
  if (g)
    for (int i = 0; i < P; ++i)
      if ((rc = change_basis(t->c[i], t->U[i], 0, st))) return t->fail(rc, t->c[i]->err.c_str());
  return DG_OK;
}

}  // namespace

extern "C" int dg_part_create(dg_ctx* const* ctxs, void* const* U, int32_t P, const int32_t* n_ghost,
                              const int32_t* ghost_src_part, const int32_t* ghost_src_elem, dg_part** out) {
  if (!out) return DG_EINVAL;
  *out = nullptr;
  std::string& e = g_setup_err;
  if (!ctxs || !U || !n_ghost || P < 1 || P > DG_PART_MAX) {
    e = "need 1..64 parts with contexts, states and ghost counts";
    return DG_EINVAL;
  }
  dg_ctx* c0 = ctxs[0];
  if (!c0) return DG_EINVAL;
  int total = 0;
  for (int i = 0; i < P; ++i) {
    dg_ctx* c = ctxs[i];
    if (c && c->dim == 2) {
      e = "parts are not built for 2D meshes";
      return DG_EUNSUPPORTED;
    }
    if (!c || c->n != c0->n || c->prec != c0->prec || c->dev != c0->dev || c->basis != c0->basis) {
      e = "parts must share degree, precision, device and storage basis";
      return DG_EINVAL;
    }
    if (n_ghost[i] < 0 || c->Erun + n_ghost[i] != c->E) {
      e = "part " + std::to_string(i) + ": n_owned + n_ghost must equal its element count";
      return DG_EINVAL;
    }
    int rc;
    if ((rc = check_state_ptr(c, U[i], "U"))) {
      e = c->err;
      return rc;
    }
    total += n_ghost[i];
  }
  if (total > 0 && (!ghost_src_part || !ghost_src_elem)) {
    e = "ghost sources missing";
    return DG_EINVAL;
  }
  std::vector<int32_t> map(4 * (size_t)total);
  int g = 0;
  for (int i = 0; i < P; ++i)
    for (int j = 0; j < n_ghost[i]; ++j, ++g) {
      const int sp = ghost_src_part[g], se = ghost_src_elem[g];
      if (sp < 0 || sp >= P || sp == i || se < 0 || se >= ctxs[sp]->Erun) {
        e = "ghost " + std::to_string(g) + ": source is not an owned element of another part";
        return DG_EINVAL;
      }
      map[4 * g] = i;
      map[4 * g + 1] = ctxs[i]->Erun + j;
      map[4 * g + 2] = sp;
      map[4 * g + 3] = se;
    }
  DeviceGuard dgd(c0->dev);
  dg_part* t = new (std::nothrow) dg_part();
  if (!t) return DG_ENOMEM;
  t->dev = c0->dev;
  t->P = P;
  t->nghost = total;
  t->words = (int)(4 * (size_t)c0->n * c0->n * c0->n * c0->rsize / 16);
  t->c.assign(ctxs, ctxs + P);
  t->U.assign(U, U + P);
  if (total) {
    cudaError_t ce = cudaMalloc(&t->map, sizeof(int32_t) * map.size());
    if (ce == cudaSuccess)
      ce = cudaMemcpy(t->map, map.data(), sizeof(int32_t) * map.size(), cudaMemcpyHostToDevice);
    if (ce != cudaSuccess) {
      cudaGetLastError();
      e = std::string("ghost map: ") + cudaGetErrorString(ce);
      delete t;
      return DG_ENOMEM;
    }
  }
  *out = t;
  return DG_OK;
}

extern "C" int dg_part_exchange(dg_part* t, uintptr_t stream) {
  if (!t) return DG_EINVAL;
  DeviceGuard g(t->dev);
  return part_exchange(t, t->U.data(), S(stream));
}

extern "C" int dg_part_step_lsrk(dg_part* t, double dt, int32_t nsteps, uintptr_t stream) {
  if (!t) return DG_EINVAL;
  if (!(dt > 0.0) || !std::isfinite(dt) || nsteps < 0) return t->fail(DG_EINVAL, "need dt > 0 and nsteps >= 0");
  DeviceGuard g(t->dev);
  return part_lsrk(t, dt, nsteps, S(stream));
}

extern "C" int dg_part_step_ader(dg_part* t, double dt, int32_t nsteps, int32_t red, uintptr_t stream) {
  if (!t) return DG_EINVAL;
  if (!(dt > 0.0) || !std::isfinite(dt) || nsteps < 0) return t->fail(DG_EINVAL, "need dt > 0 and nsteps >= 0");
  if (red < 0 || red > 3) return t->fail(DG_EUNSUPPORTED, "reduce_every must be 0, 1, 2 or 3");
  DeviceGuard g(t->dev);
  return part_ader(t, dt, nsteps, red, S(stream));
}

extern "C" int dg_part_step_hdg_ader(dg_part* t, double dt, int32_t nsteps, int32_t red, uintptr_t stream) {
  if (!t) return DG_EINVAL;
  if (!(dt > 0.0) || !std::isfinite(dt) || nsteps < 0) return t->fail(DG_EINVAL, "need dt > 0 and nsteps >= 0");
  if (red < 0 || red > 3) return t->fail(DG_EUNSUPPORTED, "reduce_every must be 0, 1, 2 or 3");
  DeviceGuard g(t->dev);
  return part_ader(t, dt, nsteps, red, S(stream), true);
}

extern "C" int dg_part_info(const dg_part* t, int32_t* n_parts, int32_t* n_ghost_total, uint64_t* exchanges) {
  if (!t) return DG_EINVAL;
  if (n_parts) *n_parts = t->P;
  if (n_ghost_total) *n_ghost_total = t->nghost;
  if (exchanges) *exchanges = t->launches;
  return DG_OK;
}

extern "C" const char* dg_part_last_error(const dg_part* t) { return t ? t->err.c_str() : ""; }

extern "C" void dg_part_destroy(dg_part* t) { delete t; }

// ---------------------------------------------------------------------------
// The 2D path (quadrilaterals): the same scheme one dimension down, with the
// state held at the Gauss points inside the steppers.  Contexts created by
// dg_mesh_setup_2d take dg_apply_operator, dg_step_lsrk, dg_step_ader
// (reduction 0 or 2), dg_tck, dg_energy, dg_norms, dg_solve_host,
// dg_set_coefficients and dg_change_basis; the other calls return
// DG_EUNSUPPORTED for them.
// ---------------------------------------------------------------------------
namespace {

int pick_epb2(int n, int bytes_per_elem, int target_threads, int max_threads) {
  int epb = target_threads / n;
  if (epb < 1) epb = 1;
  while (epb > 1 && (epb * bytes_per_elem > 200 * 1024 || epb * n > max_threads)) --epb;
  return epb;
}

int validate_mesh2(const dg_mesh2d_desc* m, std::string* err) {
  char buf[256];
  const int E = m->n_elem;
  for (int e = 0; e < E; ++e)
    for (int f = 0; f < 4; ++f) {
      const int en = m->nbr[e * 4 + f];
      if (en < -1 || en >= E) {
        snprintf(buf, sizeof buf, "nbr[%d][%d] = %d out of range", e, f, en);
        *err = buf;
        return DG_EMESH;
      }
      if (en < 0) continue;
      const int fn = m->nbr_face[e * 4 + f], o = m->orient[e * 4 + f];
      if (fn < 0 || fn >= 4 || (o != 0 && o != 1)) {
        snprintf(buf, sizeof buf, "nbr_face/orient of (%d,%d) out of range", e, f);
        *err = buf;
        return DG_EMESH;
      }
      if (m->nbr[en * 4 + fn] != e || m->nbr_face[en * 4 + fn] != f || m->orient[en * 4 + fn] != o) {
        snprintf(buf, sizeof buf, "face (%d,%d) -> (%d,%d) is not reciprocated", e, f, en, fn);
        *err = buf;
        return DG_EMESH;
      }
    }
  return DG_OK;
}

int run_setup2(dg_ctx* ctx, cudaStream_t st) {
  Setup2Params P;
  P.E = ctx->E;
  P.n = ctx->n;
  P.q = ctx->q;
  P.alpha = ctx->alpha;
  P.nodes = ctx->nodes;
  P.rho = ctx->rho;
  P.c = ctx->c;
  P.nbr = ctx->nbr;
  P.nbr_face = ctx->nbr_face;
  P.orient = ctx->orient;
  P.pts = ctx->pts;
  P.xq = ctx->xq;
  P.geoA = ctx->geoA;
  P.geoM = ctx->geoM;
  P.geoF = ctx->geoF;
  P.geoT = ctx->geoT;
  P.tstride = ctx->tstride;
  P.tstep = ctx->tstep;
  P.prec = ctx->prec;
  P.bad = ctx->bad;
  DG_CK(cudaMemsetAsync(ctx->bad, 0, sizeof(int), st), "memset");
  DG_CK(launch_setup2d(P, st), "2D set-up kernel launch");
  ctx->launches++;
  int bad = 0;
  DG_CK(cudaMemcpyAsync(&bad, ctx->bad, sizeof(int), cudaMemcpyDeviceToHost, st), "copy flag");
  DG_CK(cudaStreamSynchronize(st), "2D set-up kernel");
  if (bad) return ctx->fail(DG_EMESH, "non-positive Jacobian determinant in the mesh");
  return DG_OK;
}

int change_basis2(dg_ctx* ctx, void* U, int to_g, cudaStream_t st) {
  dg_ctx::Span span(ctx, DG_KIND_OTHER, st);
  DG_CK(g_kt2.basis[ctx->prec][ctx->n](U, ctx->E, to_g, ctx->epb_en, st), "2D basis kernel launch");
  span.done();
  ctx->launches++;
  return DG_OK;
}

Op2Params op2_params(const dg_ctx* ctx) {
  Op2Params p;
  std::memset(&p, 0, sizeof(p));
  p.nbr = ctx->nbr;
  p.nbr_face = ctx->nbr_face;
  p.orient = ctx->orient;
  p.geoA = ctx->geoA;
  p.geoM = ctx->geoM;
  p.geoF = ctx->geoF;
  p.E = ctx->E;
  return p;
}

int launch_op2(dg_ctx* ctx, const Op2Params& p, int epi, cudaStream_t st) {
  const int kind = epi == EPI_WRITE ? DG_KIND_OPERATOR : (epi == EPI_LSRK ? DG_KIND_LSRK : DG_KIND_ADER);
  dg_ctx::Span span(ctx, kind, st);
  DG_CK(g_kt2.op[ctx->prec][ctx->n](p, epi, ctx->epb_op, st), "2D operator kernel launch");
  span.done();
  ctx->launches++;
  return DG_OK;
}

int launch_tck2(dg_ctx* ctx, const void* U, void* Ubar, double dt, int red, cudaStream_t st) {
  Tck2Params p;
  std::memset(&p, 0, sizeof(p));
  p.U = U;
  p.Ubar = Ubar;
  p.geoT = ctx->geoT;
  p.geoT_stride = ctx->tstride;
  p.geo_step = ctx->tstep;
  p.E = ctx->E;
  double fact = 1.0;
  for (int j = 0; j <= ctx->n; ++j) {
    fact *= (j + 1);
    p.coef[j] = std::pow(dt, j + 1) / fact;
  }
  dg_ctx::Span span(ctx, DG_KIND_TCK, st);
  DG_CK(g_kt2.tck[ctx->prec][ctx->n](p, red, ctx->epb_tck, st), "2D predictor kernel launch");
  span.done();
  ctx->launches++;
  return DG_OK;
}

int lsrk_steps2(dg_ctx* ctx, void* U, double dt, int nsteps, cudaStream_t st) {
  int rc;
  if ((rc = ensure(ctx, &ctx->U2, "LSRK state")) || (rc = ensure(ctx, &ctx->U3, "LSRK state")) ||
      (rc = ensure(ctx, &ctx->dU, "LSRK register")))
    return rc;
  if (nsteps == 0) return DG_OK;
  if ((rc = change_basis2(ctx, U, 1, st))) return rc;
  void* const chain[6] = {U, ctx->U2, ctx->U3, ctx->U2, ctx->U3, U};
  Op2Params p = op2_params(ctx);
  for (int s = 0; s < nsteps; ++s)
    for (int st5 = 0; st5 < 5; ++st5) {
      p.U = chain[st5];
      p.Uadd = chain[st5];
      p.out = chain[st5 + 1];
      p.dU = ctx->dU;
      p.cA = kLsrkA[st5];
      p.cB = kLsrkB[st5];
      p.dt = dt;
      p.first = st5 == 0;
      if ((rc = launch_op2(ctx, p, EPI_LSRK, st))) return rc;
    }
  return change_basis2(ctx, U, 0, st);
}

int ader_steps2(dg_ctx* ctx, void* U, double dt, int nsteps, int red, cudaStream_t st) {
  int rc;
  if ((rc = ensure(ctx, &ctx->Ubar, "ADER predictor"))) return rc;
  if (nsteps == 0) return DG_OK;
  if ((rc = change_basis2(ctx, U, 1, st))) return rc;
  Op2Params p = op2_params(ctx);
  for (int s = 0; s < nsteps; ++s) {
    if ((rc = launch_tck2(ctx, U, ctx->Ubar, dt, red, st))) return rc;
    p.U = ctx->Ubar;
    p.Uadd = U;
    p.out = U;
    if ((rc = launch_op2(ctx, p, EPI_ADD, st))) return rc;
  }
  return change_basis2(ctx, U, 0, st);
}

// R = -M^-1 K U with GL states in and out (the operator works on Gauss values)
int apply2(dg_ctx* ctx, const void* U, void* R, cudaStream_t st) {
  int rc;
  if ((rc = ensure(ctx, &ctx->U2, "scratch state"))) return rc;
  DG_CK(cudaMemcpyAsync(ctx->U2, U, ctx->state_bytes(), cudaMemcpyDeviceToDevice, st), "copy");
  if ((rc = change_basis2(ctx, ctx->U2, 1, st))) return rc;
  Op2Params p = op2_params(ctx);
  p.U = ctx->U2;
  p.out = R;
  if ((rc = launch_op2(ctx, p, EPI_WRITE, st))) return rc;
  return change_basis2(ctx, R, 0, st);
}

int tck2_gl(dg_ctx* ctx, const void* U, void* Ubar, double dt, int red, cudaStream_t st) {
  int rc;
  if ((rc = ensure(ctx, &ctx->U2, "scratch state"))) return rc;
  DG_CK(cudaMemcpyAsync(ctx->U2, U, ctx->state_bytes(), cudaMemcpyDeviceToDevice, st), "copy");
  if ((rc = change_basis2(ctx, ctx->U2, 1, st))) return rc;
  if ((rc = launch_tck2(ctx, ctx->U2, Ubar, dt, red, st))) return rc;
  return change_basis2(ctx, Ubar, 0, st);
}

int energy2(dg_ctx* ctx, const void* U, double* out, cudaStream_t st) {
  int rc;
  const int blocks = (ctx->E + ctx->epb_en - 1) / ctx->epb_en;
  if ((rc = ensure_partial(ctx, blocks))) return rc;
  Energy2Params p;
  p.U = U;
  p.geoM = ctx->geoM;
  p.partial = ctx->partial;
  p.E = ctx->E;
  DG_CK(g_kt2.energy[ctx->prec][ctx->n](p, ctx->epb_en, st), "2D energy kernel launch");
  ctx->launches++;
  std::vector<double> h(blocks);
  DG_CK(cudaMemcpyAsync(h.data(), ctx->partial, sizeof(double) * blocks, cudaMemcpyDeviceToHost, st),
        "copy partials");
  DG_CK(cudaStreamSynchronize(st), "energy");
  double s = 0.0;
  for (int i = 0; i < blocks; ++i) s += h[i];
  *out = s;
  return DG_OK;
}

}  // namespace

extern "C" int dg_mesh_setup_2d(const dg_mesh2d_desc* m, int k, int prec, double alpha, const double* rho_h,
                                const double* c_h, uintptr_t stream, dg_ctx** out) {
  if (!out) return DG_EINVAL;
  *out = nullptr;
  g_setup_err.clear();
  if (!m || !m->nodes || !m->nbr || !m->nbr_face || !m->orient || m->n_elem < 1) {
    g_setup_err = "NULL mesh array or n_elem < 1";
    return DG_EINVAL;
  }
  if (k < 1 || k > DG_KMAX) {
    g_setup_err = "degree k outside [1, DG_KMAX]";
    return DG_EUNSUPPORTED;
  }
  if (m->geom_degree < 1 || m->geom_degree > DG_NMAX) {
    g_setup_err = "geometry degree outside [1, 8]";
    return DG_EUNSUPPORTED;
  }
  if (prec != DG_FP64 && prec != DG_FP32) {
    g_setup_err = "precision must be DG_FP64 or DG_FP32";
    return DG_EINVAL;
  }
  if (!(alpha >= 0.0 && alpha <= 1.0)) {
    g_setup_err = "flux_alpha outside [0, 1]";
    return DG_EINVAL;
  }
  if ((rho_h == nullptr) != (c_h == nullptr)) {
    g_setup_err = "rho and c must both be given or both be NULL";
    return DG_EINVAL;
  }
  int rc = validate_mesh2(m, &g_setup_err);
  if (rc) return rc;
  const int n = k + 1, n2 = n * n, E = m->n_elem, qc = m->geom_degree + 1;
  if (rho_h)
    for (size_t i = 0; i < (size_t)n2 * E; ++i)
      if (!(rho_h[i] > 0.0) || !(c_h[i] > 0.0) || !std::isfinite(rho_h[i]) || !std::isfinite(c_h[i])) {
        g_setup_err = "coefficients must be positive and finite";
        return DG_EINVAL;
      }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    g_setup_err = "no CUDA device";
    return DG_ECUDA;
  }
  if ((rc = init_device(dev, &g_setup_err))) return rc;
  dg_ctx* ctx = new (std::nothrow) dg_ctx();
  if (!ctx) return DG_ENOMEM;
  ctx->dim = 2;
  ctx->basis = DG_BASIS_G;
  ctx->dev = dev;
  ctx->E = ctx->Erun = E;
  ctx->k = k;
  ctx->n = n;
  ctx->q = m->geom_degree;
  ctx->prec = prec;
  ctx->alpha = alpha;
  ctx->rsize = prec == DG_FP64 ? 8 : 4;
  ctx->tstep = 2;
  ctx->tstride = geo2_stride_T(n, 2);
  cudaStream_t st = S(stream);
  auto bail = [&](int code) {
    g_setup_err = ctx->err;
    delete ctx;
    return code;
  };
  const size_t rs = ctx->rsize;
  if ((rc = ctx->alloc(&ctx->nbr, sizeof(int32_t) * 4 * E, "nbr")) ||
      (rc = ctx->alloc(&ctx->nbr_face, 4 * (size_t)E, "nbr_face")) ||
      (rc = ctx->alloc(&ctx->orient, 4 * (size_t)E, "orient")) ||
      (rc = ctx->alloc(&ctx->nodes, sizeof(double) * 2 * qc * qc * (size_t)E, "nodes")) ||
      (rc = ctx->alloc(&ctx->rho, sizeof(double) * n2 * (size_t)E, "rho")) ||
      (rc = ctx->alloc(&ctx->c, sizeof(double) * n2 * (size_t)E, "c")) ||
      (rc = ctx->alloc(&ctx->pts, sizeof(double) * 3 * DG_PTS_LEN, "points")) ||
      (rc = ctx->alloc(&ctx->xq, sizeof(double) * (DG_NMAX + 2), "geometry points")) ||
      (rc = ctx->alloc(&ctx->bad, sizeof(int), "flag")) ||
      (rc = ctx->alloc(&ctx->geoA, rs * geo2_stride_A(n) * (size_t)E, "cell metric")) ||
      (rc = ctx->alloc(&ctx->geoM, rs * geo2_stride_M(n) * (size_t)E, "mass diagonal")) ||
      (rc = ctx->alloc(&ctx->geoF, rs * geo2_stride_F(n) * (size_t)E, "face data")) ||
      (rc = ctx->alloc(&ctx->geoT, rs * (size_t)ctx->tstride * E, "predictor geometry")))
    return bail(rc);
  std::vector<double> hpts(3 * DG_PTS_LEN);
  std::memcpy(hpts.data(), g_tab.xg, sizeof(double) * DG_PTS_LEN);
  std::memcpy(hpts.data() + DG_PTS_LEN, g_tab.wg, sizeof(double) * DG_PTS_LEN);
  std::memcpy(hpts.data() + 2 * DG_PTS_LEN, g_tab.xgl, sizeof(double) * DG_PTS_LEN);
  std::vector<double> hxq(DG_NMAX + 2, 0.0);
  gauss_lobatto(qc, hxq.data());
  std::vector<double> ones(rho_h ? 0 : (size_t)n2 * E, 1.0);
  const double* rho_src = rho_h ? rho_h : ones.data();
  const double* c_src = c_h ? c_h : ones.data();
  cudaError_t ce;
#define DG_UP(dst, src, bytes)                                                            \
  if ((ce = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st)) != cudaSuccess) { \
    ctx->cuda_fail(ce, "upload");                                                         \
    return bail(DG_ECUDA);                                                                \
  }
  DG_UP(ctx->nbr, m->nbr, sizeof(int32_t) * 4 * E);
  DG_UP(ctx->nbr_face, m->nbr_face, 4 * (size_t)E);
  DG_UP(ctx->orient, m->orient, 4 * (size_t)E);
  DG_UP(ctx->nodes, m->nodes, sizeof(double) * 2 * qc * qc * (size_t)E);
  DG_UP(ctx->rho, rho_src, sizeof(double) * n2 * (size_t)E);
  DG_UP(ctx->c, c_src, sizeof(double) * n2 * (size_t)E);
  DG_UP(ctx->pts, hpts.data(), sizeof(double) * 3 * DG_PTS_LEN);
  DG_UP(ctx->xq, hxq.data(), sizeof(double) * (DG_NMAX + 2));
#undef DG_UP
  const int pi = ctx->prec;
  ctx->epb_op = pick_epb2(n, g_kt2.smem[pi][n](0), 128, g_kt2.maxthr[pi][n](0));
  ctx->epb_tck = pick_epb2(n, g_kt2.smem[pi][n](1), 128, g_kt2.maxthr[pi][n](1));
  ctx->epb_en = pick_epb2(n, g_kt2.smem[pi][n](2), 128, g_kt2.maxthr[pi][n](2));
  if ((rc = run_setup2(ctx, st))) return bail(rc);
  *out = ctx;
  return DG_OK;
}
