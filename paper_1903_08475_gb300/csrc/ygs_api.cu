// C ABI of libygs: descriptor validation, plan lifetime, and the solve /
// adjoint entry points (step 1 at create, steps 2-5 of Sect. 4.3 per solve).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>

#include "ygs_internal.h"

namespace ygs {

static thread_local std::string g_err;
static thread_local long long g_alloc_countdown = 0;  // 0: no injection

void set_error(const std::string& msg) { g_err = msg; }

void arm_alloc_injection() {
  const char* v = getenv("YGS_INJECT_ALLOC_FAILURE");
  g_alloc_countdown = v ? atoll(v) : 0;
}

cudaError_t dev_malloc(void** ptr, size_t bytes) {
  if (g_alloc_countdown > 0 && --g_alloc_countdown == 0) {
    *ptr = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMalloc(ptr, bytes);
}

namespace {

struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) ok = (cudaSetDevice(dev) == cudaSuccess);
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

ygs_status fail(ygs_status s, const std::string& msg) {
  set_error(msg);
  return s;
}

ygs_status cuda_fail(cudaError_t e, const char* what) {
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? YGS_ERR_OOM : YGS_ERR_CUDA;
}

#define API_TRY(expr)                                  \
  do {                                                 \
    cudaError_t _e = (expr);                           \
    if (_e != cudaSuccess) return cuda_fail(_e, #expr); \
  } while (0)

bool finite(double x) { return std::isfinite(x); }

void free_plan(ygs_plan* p) {
  if (!p) return;
  for (cudaEvent_t e : p->prof_events) cudaEventDestroy(e);
  for (cudaStream_t st : {p->hm_in, p->hm_out})
    if (st) {
      cudaStreamSynchronize(st);
      cudaStreamDestroy(st);
    }
  for (cudaEvent_t e : p->hm_ev)
    if (e) cudaEventDestroy(e);
  tc_free(p);
  void* bufs[] = {p->U, p->Q, p->rad, p->col_l, p->col_nat, p->chunks, p->part, p->B, p->M,
                  p->Mbar, p->Bbar, p->d_err, p->h2d_rho, p->h2d_phi, p->h2d_rho2, p->h2d_phi2,
                  p->U32, p->Q32, p->f32_field, p->part32, p->M32};
  for (void* b : bufs)
    if (b) cudaFree(b);
  delete p;
}

// Euler matrix of Eq. rottransmatrix, x = R xi.
void euler_R(const double* e, double* R) {
  double ca = cos(e[0]), sa = sin(e[0]), cb = cos(e[1]), sb = sin(e[1]), cg = cos(e[2]), sg = sin(e[2]);
  R[0] = ca * cb * cg - sa * sg;
  R[1] = sa * cb * cg + ca * sg;
  R[2] = -sb * cg;
  R[3] = -ca * cb * sg - sa * cg;
  R[4] = -sa * cb * sg + ca * cg;
  R[5] = sb * sg;
  R[6] = ca * sb;
  R[7] = sa * sb;
  R[8] = cb;
}

// Patch 1 is patch 0 turned by pi about the global z axis (R1 = diag(-1,-1,1) R0)
// on an identical local grid with identical overlap weights: then every global
// real harmonic takes the factor (-1)^m between the two patches (Sect. 4.2).
bool detect_symmetry(const ygs_plan* p) {
  if (p->n_patch != 2 || (p->flags & YGS_FLAG_NO_SYMMETRY)) return false;
  if (p->kind[0] != YGS_PATCH_LATLON || p->kind[1] != YGS_PATCH_LATLON) return false;
  if (p->nth[0] != p->nth[1] || p->nph[0] != p->nph[1]) return false;
  for (int k = 0; k < 2; ++k)
    if (p->theta_range[k] != p->theta_range[2 + k] || p->phi_range[k] != p->phi_range[2 + k]) return false;
  long long na = p->nang[0];
  if (std::memcmp(p->w_host.data(), p->w_host.data() + na, na * sizeof(double)) != 0) return false;
  double R0[9], R1[9];
  euler_R(&p->euler[0], R0);
  euler_R(&p->euler[3], R1);
  const double S[3] = {-1.0, -1.0, 1.0};
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c)
      if (fabs(R1[3 * r + c] - S[r] * R0[3 * r + c]) > 1e-13) return false;
  return true;
}

ygs_status validate_desc(const ygs_desc* d) {
  if (!d) return fail(YGS_ERR_INVALID_ARG, "desc is NULL");
  if (d->n_r < 1) return fail(YGS_ERR_INVALID_ARG, "n_r must be >= 1");
  if (!d->r_edges) return fail(YGS_ERR_INVALID_ARG, "r_edges is NULL");
  for (int i = 0; i <= d->n_r; ++i)
    if (!finite(d->r_edges[i])) return fail(YGS_ERR_INVALID_ARG, "r_edges has a non-finite value");
  if (d->r_edges[0] < 0.0) return fail(YGS_ERR_INVALID_ARG, "r_edges[0] must be >= 0");
  for (int i = 0; i < d->n_r; ++i)
    if (!(d->r_edges[i + 1] > d->r_edges[i])) return fail(YGS_ERR_INVALID_ARG, "r_edges must increase strictly");
  if (d->n_patch < 1 || d->n_patch > kMaxPatch)
    return fail(YGS_ERR_INVALID_ARG, "n_patch must be in [1, " + std::to_string(kMaxPatch) + "]");
  if (!d->euler || !d->n_theta || !d->n_phi || !d->theta_range || !d->phi_range || !d->overlap_w)
    return fail(YGS_ERR_INVALID_ARG, "a patch array is NULL");
  long long total = 0;
  const double pi = 3.14159265358979323846;
  for (int g = 0; g < d->n_patch; ++g) {
    for (int k = 0; k < 3; ++k)
      if (!finite(d->euler[3 * g + k])) return fail(YGS_ERR_INVALID_ARG, "non-finite Euler angle");
    if (d->n_theta[g] < 1 || d->n_phi[g] < 1) return fail(YGS_ERR_INVALID_ARG, "n_theta and n_phi must be >= 1");
    double t0 = d->theta_range[2 * g], t1 = d->theta_range[2 * g + 1];
    double p0 = d->phi_range[2 * g], p1 = d->phi_range[2 * g + 1];
    if (!finite(t0) || !finite(t1) || !finite(p0) || !finite(p1))
      return fail(YGS_ERR_INVALID_ARG, "non-finite patch extent");
    const int kind = d->patch_kind ? d->patch_kind[g] : YGS_PATCH_LATLON;
    if (kind == YGS_PATCH_GNOMONIC) {
      // xi and eta strictly inside (-pi/2, pi/2), where tan is finite
      const double h = 0.5 * pi - 1e-6;
      if (t0 < -h || t1 > h || !(t1 > t0) || p0 < -h || p1 > h || !(p1 > p0))
        return fail(YGS_ERR_INVALID_ARG, "a gnomonic patch's xi and eta ranges must satisfy -pi/2 < lo < hi < pi/2");
    } else if (kind == YGS_PATCH_LATLON) {
      if (t0 < -1e-12 || t1 > pi + 1e-12 || !(t1 > t0)) return fail(YGS_ERR_INVALID_ARG, "theta_range must satisfy 0 <= lo < hi <= pi");
      if (!(p1 > p0) || p1 - p0 > 2 * pi + 1e-12) return fail(YGS_ERR_INVALID_ARG, "phi_range must satisfy lo < hi <= lo + 2 pi");
    } else {
      return fail(YGS_ERR_INVALID_ARG, "unknown patch kind");
    }
    long long na = (long long)d->n_theta[g] * d->n_phi[g];
    if (na > (1LL << 30)) return fail(YGS_ERR_INVALID_ARG, "too many angular cells in one patch");
    total += na;
  }
  for (long long a = 0; a < total; ++a)
    if (!finite(d->overlap_w[a])) return fail(YGS_ERR_INVALID_ARG, "non-finite overlap weight");
  if (d->l_max < 0 || d->l_max > kMaxLmax)
    return fail(YGS_ERR_INVALID_ARG, "l_max must be in [0, " + std::to_string(kMaxLmax) + "]");
  if (!finite(d->G)) return fail(YGS_ERR_INVALID_ARG, "G must be finite");
  if (d->eval != YGS_EVAL_UPPER_VERTEX && d->eval != YGS_EVAL_CELL_CENTRE) return fail(YGS_ERR_INVALID_ARG, "bad eval");
  if (d->precision < YGS_FP64 || d->precision > YGS_FP64_EMU) return fail(YGS_ERR_INVALID_ARG, "bad precision");
  if (d->flags & ~(YGS_FLAG_NO_SYMMETRY | YGS_FLAG_AUTOTUNE | YGS_FLAG_CTA_PAIRS)) return fail(YGS_ERR_INVALID_ARG, "unknown flag bits");
  if ((long long)d->n_r * total > (1LL << 40)) return fail(YGS_ERR_INVALID_ARG, "field too large");
  return YGS_OK;
}

constexpr int kProfCap = 4096;
constexpr int kPhases = 4;

// Returns the kPhases + 1 events of the next recorded call, or nullptr when profiling is off / full.
cudaEvent_t* prof_slot(ygs_plan* p) {
  if (!p->profiling || p->prof_used >= kProfCap) return nullptr;
  size_t need = (size_t)(p->prof_used + 1) * (kPhases + 1);
  while (p->prof_events.size() < need) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    p->prof_events.push_back(e);
  }
  return &p->prof_events[(size_t)p->prof_used++ * (kPhases + 1)];
}

// Per-device pool of worker streams for batched solves (created on first use,
// kept until process exit).  Events fork the caller's stream onto the workers
// and join them back, which also works under CUDA stream capture.
constexpr int kPoolStreams = 8;
struct StreamPool {
  cudaStream_t s[kPoolStreams];
  cudaEvent_t fork;
  cudaEvent_t join[kPoolStreams];
};
std::mutex g_pool_mu;
std::map<int, StreamPool*> g_pools;

StreamPool* get_pool(int device, ygs_status* st) {
  std::lock_guard<std::mutex> lk(g_pool_mu);
  auto it = g_pools.find(device);
  if (it != g_pools.end()) return it->second;
  StreamPool* P = new (std::nothrow) StreamPool();
  if (!P) {
    *st = fail(YGS_ERR_OOM, "host allocation failed");
    return nullptr;
  }
  cudaError_t e = cudaEventCreateWithFlags(&P->fork, cudaEventDisableTiming);
  for (int k = 0; k < kPoolStreams && e == cudaSuccess; ++k) {
    e = cudaStreamCreateWithFlags(&P->s[k], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&P->join[k], cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    *st = cuda_fail(e, "stream pool");
    return nullptr;
  }
  g_pools[device] = P;
  return P;
}

bool aligned16(const void* ptr) { return ((uintptr_t)ptr & 15u) == 0; }

ygs_status check_field(const ygs_plan* p, const void* a, const void* b) {
  if (!p) return fail(YGS_ERR_INVALID_ARG, "plan is NULL");
  if (!a || !b) return fail(YGS_ERR_INVALID_ARG, "field pointer is NULL");
  if (!aligned16(a) || !aligned16(b)) return fail(YGS_ERR_INVALID_ARG, "field pointers must be 16-byte aligned");
  const char* ca = (const char*)a;
  const char* cb = (const char*)b;
  size_t bytes = (size_t)p->n_cells * sizeof(double);
  if (ca < cb + bytes && cb < ca + bytes) return fail(YGS_ERR_INVALID_ARG, "input and output fields overlap");
  return YGS_OK;
}

}  // namespace
}  // namespace ygs

namespace ygs {
// The checked build's site names, by BoundsSite.
const char* bounds_site_name(int site) {
  static const char* const names[kSiteBoundsSites] = {
      "none", "field pass FP16: rho load", "field pass FP16: slice store", "field pass FP16: factor store",
      "field pass FP16: monopole weight load", "field pass BF16/TF32: rho load", "field pass BF16/TF32: slice store",
      "radial scan: partial load", "radial scan: B/M store", "radial scan: M slice store", "M slicing: M load",
      "M slicing: slice store", "contraction epilogue: Phi store", "contraction epilogue: partial store",
      "contraction producer: factor row", "FP64 projection: field load", "FP64 projection: weight load",
      "FP64 projection: partial store", "FP64 synthesis: moment load", "FP64 synthesis: weight load",
      "FP64 synthesis: Phi store", "FP64 radial scan", "FP64 adjoint scan", "FP64-accurate field pass: rho load",
      "FP64-accurate field pass: slice store", "FP64-accurate radial scan"};
  return site > 0 && site < kSiteBoundsSites ? names[site] : "unknown site";
}
}  // namespace ygs

using namespace ygs;

extern "C" {

const char* ygs_status_string(ygs_status s) {
  switch (s) {
    case YGS_OK: return "YGS_OK";
    case YGS_ERR_INVALID_ARG: return "YGS_ERR_INVALID_ARG";
    case YGS_ERR_OOM: return "YGS_ERR_OOM";
    case YGS_ERR_CUDA: return "YGS_ERR_CUDA";
    case YGS_ERR_UNSUPPORTED: return "YGS_ERR_UNSUPPORTED";
    case YGS_ERR_NUMERIC: return "YGS_ERR_NUMERIC";
    case YGS_ERR_TIMEOUT: return "YGS_ERR_TIMEOUT";
    case YGS_ERR_BOUNDS: return "YGS_ERR_BOUNDS";
  }
  return "YGS_ERR_UNKNOWN";
}

const char* ygs_last_error(void) { return g_err.c_str(); }

ygs_status ygs_create(const ygs_desc* d, int device, ygs_plan** out) {
  if (!out) return fail(YGS_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  ygs_status st = validate_desc(d);
  if (st != YGS_OK) return st;
  int ndev = 0;
  API_TRY(cudaGetDeviceCount(&ndev));
  if (device < 0 || device >= ndev) return fail(YGS_ERR_INVALID_ARG, "bad device index");
  DeviceGuard guard(device);
  if (!guard.ok) return fail(YGS_ERR_CUDA, "cudaSetDevice failed");
  arm_alloc_injection();

  ygs_plan* p = new (std::nothrow) ygs_plan();
  if (!p) return fail(YGS_ERR_OOM, "host allocation failed");
  p->device = device;
  p->n_r = d->n_r;
  p->n_patch = d->n_patch;
  p->l_max = d->l_max;
  p->K = (d->l_max + 1) * (d->l_max + 1);
  p->precision = d->precision;
  p->eval = d->eval;
  p->flags = d->flags;
  p->G = d->G;
  p->edges.assign(d->r_edges, d->r_edges + d->n_r + 1);
  p->euler.assign(d->euler, d->euler + 3 * d->n_patch);
  p->theta_range.assign(d->theta_range, d->theta_range + 2 * d->n_patch);
  p->phi_range.assign(d->phi_range, d->phi_range + 2 * d->n_patch);
  p->nth.assign(d->n_theta, d->n_theta + d->n_patch);
  p->nph.assign(d->n_phi, d->n_phi + d->n_patch);
  if (d->patch_kind)
    p->kind.assign(d->patch_kind, d->patch_kind + d->n_patch);
  else
    p->kind.assign(d->n_patch, (int)YGS_PATCH_LATLON);
  long long acc = 0;
  for (int g = 0; g < p->n_patch; ++g) {
    p->nang.push_back((long long)p->nth[g] * p->nph[g]);
    p->ang_off.push_back(acc);
    p->fld_off.push_back(acc * p->n_r);
    acc += p->nang.back();
  }
  p->nang_total = acc;
  p->n_cells = acc * p->n_r;
  p->w_host.assign(d->overlap_w, d->overlap_w + acc);
  p->symmetric = detect_symmetry(p);
  p->n_wpatch = p->symmetric ? 1 : p->n_patch;
  p->nang_wtotal = p->symmetric ? p->nang[0] : acc;
  for (int g = 0; g < p->n_patch; ++g) {
    p->pt.fld_off[g] = p->fld_off[g];
    p->pt.nang[g] = p->nang[g];
    p->pt.ang_off[g] = p->symmetric ? 0 : p->ang_off[g];
  }
  p->pt.n_cells = p->n_cells;
  p->pt.w_rows = p->nang_wtotal;
  // internal column order: even m first when the symmetry is used
  p->col_perm.clear();
  if (p->symmetric) {
    for (int par = 0; par < 2; ++par)
      for (int c = 0; c < p->K; ++c) {
        int l = 0;
        while ((l + 1) * (l + 1) <= c) ++l;
        int m = (c - l * l + 1) / 2;
        if ((m & 1) == par) p->col_perm.push_back(c);
      }
    p->K_even = 0;
    for (int c : p->col_perm) {
      int l = 0;
      while ((l + 1) * (l + 1) <= c) ++l;
      if ((((c - l * l + 1) / 2) & 1) == 0) ++p->K_even;
    }
  } else {
    for (int c = 0; c < p->K; ++c) p->col_perm.push_back(c);
    p->K_even = p->K;
  }

  // split-K chunks over the stored patches' angular cells
  int sms = 148;
  {
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) == cudaSuccess) sms = prop.multiProcessorCount;
  }
  const int BMt = 64, BNt = 64, BKt = 16;
  long long tiles = (long long)((p->n_r + BMt - 1) / BMt) *
                    ((p->K_even + BNt - 1) / BNt + (p->K - p->K_even + BNt - 1) / BNt);
  long long want = std::max(1LL, (4LL * sms + tiles - 1) / tiles);
  std::vector<Chunk> chunks;
  for (int g = 0; g < p->n_wpatch; ++g) {
    long long na = p->nang[g];
    long long sg = std::max(1LL, (want * na + p->nang_wtotal - 1) / p->nang_wtotal);
    sg = std::min(sg, std::max(1LL, na / (8 * BKt)));
    long long len = (na + sg - 1) / sg;
    len = (len + BKt - 1) / BKt * BKt;
    for (long long a0 = 0; a0 < na; a0 += len) chunks.push_back(Chunk{g, (int)a0, (int)std::min(na, a0 + len), 0});
  }
  p->S = (int)chunks.size();

  auto fail_free = [&](ygs_status s) {
    free_plan(p);
    return s;
  };
  auto al = [&](void** ptr, size_t bytes) -> cudaError_t { return dev_malloc(ptr, std::max<size_t>(bytes, 16)); };
  size_t wbytes = (size_t)p->nang_wtotal * p->K * sizeof(double);
  size_t nk = (size_t)p->n_r * p->K * sizeof(double);
  cudaError_t e;
  if ((e = al((void**)&p->U, wbytes)) != cudaSuccess) return fail_free(cuda_fail(e, "cudaMalloc U"));
  if ((e = al((void**)&p->Q, wbytes)) != cudaSuccess) return fail_free(cuda_fail(e, "cudaMalloc Q"));
  if ((e = al((void**)&p->rad, 4 * (size_t)(p->l_max + 1) * p->n_r * sizeof(double))) != cudaSuccess)
    return fail_free(cuda_fail(e, "cudaMalloc rad"));
  if ((e = al((void**)&p->col_l, p->K * sizeof(int))) != cudaSuccess) return fail_free(cuda_fail(e, "cudaMalloc col_l"));
  if ((e = al((void**)&p->col_nat, p->K * sizeof(int))) != cudaSuccess) return fail_free(cuda_fail(e, "cudaMalloc col_nat"));
  if ((e = al((void**)&p->chunks, chunks.size() * sizeof(Chunk))) != cudaSuccess)
    return fail_free(cuda_fail(e, "cudaMalloc chunks"));
  if ((e = al((void**)&p->part, (size_t)p->S * nk)) != cudaSuccess) return fail_free(cuda_fail(e, "cudaMalloc part"));
  if ((e = al((void**)&p->B, nk)) != cudaSuccess) return fail_free(cuda_fail(e, "cudaMalloc B"));
  if ((e = al((void**)&p->M, nk)) != cudaSuccess) return fail_free(cuda_fail(e, "cudaMalloc M"));
  if ((e = al((void**)&p->Mbar, nk)) != cudaSuccess) return fail_free(cuda_fail(e, "cudaMalloc Mbar"));
  if ((e = al((void**)&p->Bbar, nk)) != cudaSuccess) return fail_free(cuda_fail(e, "cudaMalloc Bbar"));
  if ((e = al((void**)&p->d_err, sizeof(int))) != cudaSuccess) return fail_free(cuda_fail(e, "cudaMalloc err"));
  if ((e = cudaMemset(p->d_err, 0, sizeof(int))) != cudaSuccess) return fail_free(cuda_fail(e, "cudaMemset err"));
  if ((e = cudaMemcpy(p->chunks, chunks.data(), chunks.size() * sizeof(Chunk), cudaMemcpyHostToDevice)) != cudaSuccess)
    return fail_free(cuda_fail(e, "cudaMemcpy chunks"));
  p->weight_bytes = 2LL * wbytes;
  p->work_bytes = (long long)(p->S + 4) * nk;

  st = build_weights(p);
  if (st != YGS_OK) return fail_free(st);
  // load what ygs_solve_static runs, so that its first call allocates nothing
  if ((e = preload_fp64_kernels()) != cudaSuccess) return fail_free(cuda_fail(e, "loading the FP64 kernels"));
  if ((e = prepare_static_scratch()) != cudaSuccess)
    return fail_free(cuda_fail(e, "making the static scratch array resident"));
  if (p->precision == YGS_BF16X6 || p->precision == YGS_BF16X3 || p->precision == YGS_FP16X3 ||
      p->precision == YGS_TF32X3 || p->precision == YGS_FP64_EMU) {
    if (p->n_r > 65535) return fail_free(fail(YGS_ERR_UNSUPPORTED, "split precision supports n_r <= 65535"));
    p->tc_nsl = (p->precision == YGS_FP64_EMU) ? 6 : ((p->precision == YGS_BF16X6) ? 3 : 2);
    p->tc_fp16 = (p->precision == YGS_FP16X3) ? 1 : 0;
    p->tc_tf32 = (p->precision == YGS_TF32X3) ? 1 : 0;
    p->tc_emu = (p->precision == YGS_FP64_EMU) ? 1 : 0;
    st = tc_setup(p, sms);
    if (st != YGS_OK) return fail_free(st);
  }
  if (p->precision == YGS_FP32) {
    const size_t wn = (size_t)p->nang_wtotal * p->K, kn = (size_t)p->n_r * p->K;
    if ((e = al((void**)&p->U32, wn * sizeof(float))) != cudaSuccess ||
        (e = al((void**)&p->Q32, wn * sizeof(float))) != cudaSuccess ||
        (e = al((void**)&p->f32_field, (size_t)p->n_cells * sizeof(float))) != cudaSuccess ||
        (e = al((void**)&p->part32, (size_t)p->S * kn * sizeof(float))) != cudaSuccess ||
        (e = al((void**)&p->M32, kn * sizeof(float))) != cudaSuccess)
      return fail_free(cuda_fail(e, "cudaMalloc FP32 operands"));
    if ((e = launch_to_f32(p->U, p->U32, (long long)wn, false, 0)) != cudaSuccess ||
        (e = launch_to_f32(p->Q, p->Q32, (long long)wn, false, 0)) != cudaSuccess ||
        (e = cudaDeviceSynchronize()) != cudaSuccess)
      return fail_free(cuda_fail(e, "FP32 weights"));
    p->weight_bytes += (long long)(2 * wn * sizeof(float));
    p->work_bytes += (long long)(((size_t)p->n_cells + (size_t)(p->S + 1) * kn) * sizeof(float));
  }
  *out = p;
  return YGS_OK;
}

ygs_status ygs_destroy(ygs_plan* p) {
  if (!p) return YGS_OK;
  DeviceGuard guard(p->device);
  cudaDeviceSynchronize();
  free_plan(p);
  return YGS_OK;
}

ygs_status ygs_get_info(const ygs_plan* p, ygs_info* info) {
  if (!p || !info) return fail(YGS_ERR_INVALID_ARG, "NULL argument");
  info->n_r = p->n_r;
  info->n_patch = p->n_patch;
  info->l_max = p->l_max;
  info->K = p->K;
  info->n_ang = p->nang_total;
  info->n_cells = p->n_cells;
  info->precision = p->precision;
  info->symmetric = p->symmetric ? 1 : 0;
  info->split_k = p->tc_nsl ? p->tc_S : p->S;
  info->weight_bytes = p->weight_bytes;
  info->work_bytes = p->work_bytes;
  info->fp64_split_k = p->S;
  info->static_scratch_bytes = static_scratch_bytes(p);
  info->cta_pairs = p->tc_pairs > 0 ? 1 : 0;
  info->synth_tile_shells = p->tc_nsl ? p->tc_N : 0;
  return YGS_OK;
}

ygs_status ygs_solve(ygs_plan* p, const double* d_rho, double* d_phi, void* stream) {
  ygs_status st = check_field(p, d_rho, d_phi);
  if (st != YGS_OK) return st;
  DeviceGuard guard(p->device);
  if (!guard.ok) return fail(YGS_ERR_CUDA, "cudaSetDevice failed");
  cudaStream_t s = (cudaStream_t)stream;
  p->last_stream = s;
  cudaEvent_t* ev = prof_slot(p);
  if (ev) API_TRY(cudaEventRecord(ev[0], s));
  if (p->tc_nsl) {
    API_TRY(tc_field_slices(p, d_rho, s));
    if (ev) API_TRY(cudaEventRecord(ev[1], s));
    API_TRY(tc_project(p, s));
    if (ev) API_TRY(cudaEventRecord(ev[2], s));
    API_TRY(tc_scan(p, s));
    if (ev) API_TRY(cudaEventRecord(ev[3], s));
    API_TRY(tc_synthesize(p, d_phi, s));
  } else {
    if (p->precision == YGS_FP32) {
      API_TRY(solve_fp32(p, d_rho, d_phi, s, ev));
    } else {
      if (ev) API_TRY(cudaEventRecord(ev[1], s));
      API_TRY(launch_project_fp64(p, d_rho, p->U, p->part, s));
      if (ev) API_TRY(cudaEventRecord(ev[2], s));
      API_TRY(launch_scan_fwd(p, p->part, p->S, p->B, p->M, s));
      if (ev) API_TRY(cudaEventRecord(ev[3], s));
      API_TRY(launch_synth_fp64(p, p->M, p->Q, d_phi, s));
    }
  }
  if (ev) API_TRY(cudaEventRecord(ev[4], s));
  return YGS_OK;
}

ygs_status ygs_solve_host(ygs_plan* p, const double* h_rho, double* h_phi, void* stream) {
  if (!p || !h_rho || !h_phi) return fail(YGS_ERR_INVALID_ARG, "NULL argument");
  DeviceGuard guard(p->device);
  size_t bytes = (size_t)p->n_cells * sizeof(double);
  if (!p->h2d_rho) API_TRY(dev_malloc((void**)&p->h2d_rho, bytes));
  if (!p->h2d_phi) API_TRY(dev_malloc((void**)&p->h2d_phi, bytes));
  cudaStream_t s = (cudaStream_t)stream;
  API_TRY(cudaMemcpyAsync(p->h2d_rho, h_rho, bytes, cudaMemcpyHostToDevice, s));
  ygs_status st = ygs_solve(p, p->h2d_rho, p->h2d_phi, stream);
  if (st != YGS_OK) return st;
  API_TRY(cudaMemcpyAsync(h_phi, p->h2d_phi, bytes, cudaMemcpyDeviceToHost, s));
  API_TRY(cudaStreamSynchronize(s));
  return YGS_OK;
}

ygs_status ygs_solve_host_many(ygs_plan* p, int n, const double* const* h_rho, double* const* h_phi,
                               void* stream) {
  if (!p || n < 0 || (n > 0 && (!h_rho || !h_phi))) return fail(YGS_ERR_INVALID_ARG, "NULL argument or n < 0");
  for (int k = 0; k < n; ++k)
    if (!h_rho[k] || !h_phi[k]) return fail(YGS_ERR_INVALID_ARG, "NULL host buffer");
  if (n == 0) return YGS_OK;
  DeviceGuard guard(p->device);
  const size_t bytes = (size_t)p->n_cells * sizeof(double);
  double** rho[2] = {&p->h2d_rho, &p->h2d_rho2};
  double** phi[2] = {&p->h2d_phi, &p->h2d_phi2};
  for (int b = 0; b < 2; ++b) {
    if (!*rho[b]) API_TRY(dev_malloc((void**)rho[b], bytes));
    if (!*phi[b]) API_TRY(dev_malloc((void**)phi[b], bytes));
  }
  if (!p->hm_in) API_TRY(cudaStreamCreateWithFlags(&p->hm_in, cudaStreamNonBlocking));
  if (!p->hm_out) API_TRY(cudaStreamCreateWithFlags(&p->hm_out, cudaStreamNonBlocking));
  for (cudaEvent_t& e : p->hm_ev)
    if (!e) API_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  cudaEvent_t start = p->hm_ev[0], *ev_in = p->hm_ev + 1, *ev_comp = p->hm_ev + 3, *ev_out = p->hm_ev + 5;
  cudaStream_t s = (cudaStream_t)stream, in = p->hm_in, out = p->hm_out;
  // the copy streams start after the work already queued on `stream`
  API_TRY(cudaEventRecord(start, s));
  API_TRY(cudaStreamWaitEvent(in, start, 0));
  API_TRY(cudaStreamWaitEvent(out, start, 0));
  for (int k = 0; k < n; ++k) {
    const int b = k & 1;
    // upload field k into staging pair b once solve k - 2 has read it
    if (k >= 2) API_TRY(cudaStreamWaitEvent(in, ev_comp[b], 0));
    API_TRY(cudaMemcpyAsync(*rho[b], h_rho[k], bytes, cudaMemcpyHostToDevice, in));
    API_TRY(cudaEventRecord(ev_in[b], in));
    // solve k once its input is in and the read-back of solve k - 2 has left pair b
    API_TRY(cudaStreamWaitEvent(s, ev_in[b], 0));
    if (k >= 2) API_TRY(cudaStreamWaitEvent(s, ev_out[b], 0));
    ygs_status st = ygs_solve(p, *rho[b], *phi[b], stream);
    if (st != YGS_OK) return st;
    API_TRY(cudaEventRecord(ev_comp[b], s));
    // read Phi_k back while solve k + 1 runs
    API_TRY(cudaStreamWaitEvent(out, ev_comp[b], 0));
    API_TRY(cudaMemcpyAsync(h_phi[k], *phi[b], bytes, cudaMemcpyDeviceToHost, out));
    API_TRY(cudaEventRecord(ev_out[b], out));
  }
  // the read-back stream is in order: its last copy ends the batch
  API_TRY(cudaStreamWaitEvent(s, ev_out[(n - 1) & 1], 0));
  API_TRY(cudaStreamSynchronize(s));
  return YGS_OK;
}

ygs_status ygs_solve_batched(int n, ygs_plan* const* plans, const double* const* d_rho, double* const* d_phi,
                             void* stream) {
  if (n < 0 || (n > 0 && (!plans || !d_rho || !d_phi))) return fail(YGS_ERR_INVALID_ARG, "bad batch arrays");
  if (n == 0) return YGS_OK;
  const int dev = plans[0] ? plans[0]->device : 0;
  for (int b = 0; b < n; ++b) {
    ygs_status st = check_field(plans[b], d_rho[b], d_phi[b]);
    if (st != YGS_OK) return st;
    if (plans[b]->device != dev) return fail(YGS_ERR_INVALID_ARG, "all plans of a batch must share one device");
  }
  if (n == 1) return ygs_solve(plans[0], d_rho[0], d_phi[0], stream);
  DeviceGuard guard(dev);
  ygs_status st = YGS_OK;
  StreamPool* P = get_pool(dev, &st);
  if (!P) return st;
  cudaStream_t s = (cudaStream_t)stream;
  API_TRY(cudaEventRecord(P->fork, s));
  // fields of one plan share its workspaces: they go to one worker stream, in order
  std::map<const ygs_plan*, int> lane;
  int next = 0;
  bool used[kPoolStreams] = {false};
  for (int b = 0; b < n; ++b) {
    auto it = lane.find(plans[b]);
    int k = (it != lane.end()) ? it->second : (lane[plans[b]] = (next++ % kPoolStreams));
    if (!used[k]) {
      API_TRY(cudaStreamWaitEvent(P->s[k], P->fork, 0));
      used[k] = true;
    }
    st = ygs_solve(plans[b], d_rho[b], d_phi[b], (void*)P->s[k]);
    if (st != YGS_OK) return st;
    plans[b]->last_stream = s;
  }
  for (int k = 0; k < kPoolStreams; ++k)
    if (used[k]) {
      API_TRY(cudaEventRecord(P->join[k], P->s[k]));
      API_TRY(cudaStreamWaitEvent(s, P->join[k], 0));
    }
  return YGS_OK;
}

struct ygs_batch {
  int device = 0;
  std::vector<ygs_plan*> plans;
  std::vector<int> split, fp64;  // indices into plans
  TcBatch tc;
};

ygs_status ygs_batch_create(int n, ygs_plan* const* plans, ygs_batch** out) {
  if (!out) return fail(YGS_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (n < 1 || n > 1024 || !plans) return fail(YGS_ERR_INVALID_ARG, "a batch holds 1 to 1024 plans");
  std::map<const ygs_plan*, int> seen;
  for (int k = 0; k < n; ++k) {
    if (!plans[k]) return fail(YGS_ERR_INVALID_ARG, "plan is NULL");
    if (plans[k]->device != plans[0]->device) return fail(YGS_ERR_INVALID_ARG, "all plans of a batch must share one device");
    if (seen.count(plans[k])) return fail(YGS_ERR_INVALID_ARG, "a plan may appear once in a batch (its workspaces serve one field)");
    seen[plans[k]] = k;
  }
  ygs_batch* b = new (std::nothrow) ygs_batch;
  if (!b) return fail(YGS_ERR_OOM, "host allocation failed");
  b->device = plans[0]->device;
  b->plans.assign(plans, plans + n);
  std::vector<ygs_plan*> sp;
  for (int k = 0; k < n; ++k) {
    if (plans[k]->tc_nsl) {
      b->split.push_back(k);
      sp.push_back(plans[k]);
    } else {
      b->fp64.push_back(k);
    }
  }
  DeviceGuard guard(b->device);
  if (!guard.ok) {
    delete b;
    return fail(YGS_ERR_CUDA, "cudaSetDevice failed");
  }
  ygs_status st = tc_batch_build(&b->tc, sp);
  if (st != YGS_OK) {
    tc_batch_free(&b->tc);
    delete b;
    return st;
  }
  *out = b;
  return YGS_OK;
}

ygs_status ygs_batch_destroy(ygs_batch* b) {
  if (!b) return YGS_OK;
  DeviceGuard guard(b->device);
  cudaDeviceSynchronize();
  tc_batch_free(&b->tc);
  delete b;
  return YGS_OK;
}

ygs_status ygs_batch_solve(ygs_batch* b, const double* const* d_rho, double* const* d_phi, void* stream) {
  if (!b || !d_rho || !d_phi) return fail(YGS_ERR_INVALID_ARG, "NULL argument");
  const int n = (int)b->plans.size();
  for (int k = 0; k < n; ++k) {
    ygs_status st = check_field(b->plans[k], d_rho[k], d_phi[k]);
    if (st != YGS_OK) return st;
  }
  DeviceGuard guard(b->device);
  if (!guard.ok) return fail(YGS_ERR_CUDA, "cudaSetDevice failed");
  cudaStream_t s = (cudaStream_t)stream;
  // per operand kind: the field slices, the projection, the scans (and M
  // slicing) and the synthesis of all its members, one grouped launch each
  auto member_fields = [&](const TcBatchGroup& G) {
    std::vector<const double*> rho;
    for (const ygs_plan* m : G.members)
      for (int k : b->split)
        if (b->plans[k] == m) rho.push_back(d_rho[k]);
    return rho;
  };
  for (const TcBatchGroup& G : b->tc.groups) {
    const std::vector<const double*> rho = member_fields(G);
    API_TRY(tc_batch_field(G, rho.data(), s));
  }
  for (const TcBatchGroup& G : b->tc.groups) API_TRY(tc_batch_project(G, s));
  for (const TcBatchGroup& G : b->tc.groups) API_TRY(tc_batch_scan(G, s));
  for (const TcBatchGroup& G : b->tc.groups) {
    std::vector<double*> phi;
    for (const ygs_plan* m : G.members)
      for (int k : b->split)
        if (b->plans[k] == m) phi.push_back(d_phi[k]);
    API_TRY(tc_batch_synthesize(G, phi.data(), s));
  }
  for (int k : b->fp64) {
    ygs_status st = ygs_solve(b->plans[k], d_rho[k], d_phi[k], stream);
    if (st != YGS_OK) return st;
  }
  for (ygs_plan* p : b->plans) p->last_stream = s;
  return YGS_OK;
}

int ygs_batch_launches(const ygs_batch* b) {
  if (!b) return 0;
  int n = 0;
  // per operand kind: field slices, projection, scan (+ M slicing), synthesis
  for (const TcBatchGroup& G : b->tc.groups) n += (G.fp16 || G.emu) ? 5 : 4;
  n += 3 * (int)b->fp64.size();
  return n;
}

ygs_status ygs_backward(ygs_plan* p, const double* d_gphi, double* d_grho, void* stream) {
  ygs_status st = check_field(p, d_gphi, d_grho);
  if (st != YGS_OK) return st;
  DeviceGuard guard(p->device);
  if (!guard.ok) return fail(YGS_ERR_CUDA, "cudaSetDevice failed");
  cudaStream_t s = (cudaStream_t)stream;
  p->last_stream = s;
  cudaEvent_t* ev = prof_slot(p);
  if (ev) API_TRY(cudaEventRecord(ev[0], s));
  if (p->tc_nsl) {
    API_TRY(tc_backward(p, d_gphi, d_grho, s, ev));
    if (ev) API_TRY(cudaEventRecord(ev[4], s));
    return YGS_OK;
  }
  if (ev) API_TRY(cudaEventRecord(ev[1], s));
  API_TRY(launch_project_fp64(p, d_gphi, p->Q, p->part, s));
  if (ev) API_TRY(cudaEventRecord(ev[2], s));
  API_TRY(launch_scan_adj(p, p->part, p->S, p->Bbar, s));
  if (ev) API_TRY(cudaEventRecord(ev[3], s));
  API_TRY(launch_synth_fp64(p, p->Bbar, p->U, d_grho, s));
  if (ev) API_TRY(cudaEventRecord(ev[4], s));
  return YGS_OK;
}

ygs_status ygs_project_partial(ygs_plan* p, const double* d_rho, int chunk_begin, int chunk_end, double* d_B,
                               void* stream) {
  if (!p || !d_rho || !d_B) return fail(YGS_ERR_INVALID_ARG, "NULL argument");
  if (!aligned16(d_rho) || !aligned16(d_B)) return fail(YGS_ERR_INVALID_ARG, "pointers must be 16-byte aligned");
  if (chunk_begin < 0 || chunk_begin > chunk_end || chunk_end > p->S)
    return fail(YGS_ERR_INVALID_ARG, "chunk range must satisfy 0 <= begin <= end <= fp64_split_k (" +
                                         std::to_string(p->S) + ")");
  DeviceGuard guard(p->device);
  if (!guard.ok) return fail(YGS_ERR_CUDA, "cudaSetDevice failed");
  cudaStream_t s = (cudaStream_t)stream;
  p->last_stream = s;
  if (chunk_begin == chunk_end) {
    API_TRY(cudaMemsetAsync(d_B, 0, (size_t)p->n_r * p->K * sizeof(double), s));
    return YGS_OK;
  }
  API_TRY(launch_project_fp64_chunks(p, d_rho, p->U, p->part, chunk_begin, chunk_end, s));
  API_TRY(launch_sum_partials(p, p->part, chunk_end - chunk_begin, p->B, s));
  API_TRY(launch_unpermute(p, p->B, d_B, s));
  return YGS_OK;
}

ygs_status ygs_finish_from_moments(ygs_plan* p, const double* d_B, double* d_phi, void* stream) {
  if (!p || !d_B || !d_phi) return fail(YGS_ERR_INVALID_ARG, "NULL argument");
  if (!aligned16(d_B) || !aligned16(d_phi)) return fail(YGS_ERR_INVALID_ARG, "pointers must be 16-byte aligned");
  const char* cb = (const char*)d_B;
  const char* cp = (const char*)d_phi;
  const size_t bb = (size_t)p->n_r * p->K * sizeof(double), pb = (size_t)p->n_cells * sizeof(double);
  if (cb < cp + pb && cp < cb + bb) return fail(YGS_ERR_INVALID_ARG, "B and Phi overlap");
  DeviceGuard guard(p->device);
  if (!guard.ok) return fail(YGS_ERR_CUDA, "cudaSetDevice failed");
  cudaStream_t s = (cudaStream_t)stream;
  p->last_stream = s;
  API_TRY(launch_permute(p, d_B, p->part, s));
  API_TRY(launch_scan_fwd(p, p->part, 1, p->B, p->M, s));
  API_TRY(launch_synth_fp64(p, p->M, p->Q, d_phi, s));
  return YGS_OK;
}

ygs_status ygs_get_moments(ygs_plan* p, double* d_B, double* d_M, void* stream) {
  if (!p) return fail(YGS_ERR_INVALID_ARG, "plan is NULL");
  DeviceGuard guard(p->device);
  cudaStream_t s = (cudaStream_t)stream;
  if (p->tc_emu) {
    if (d_B) API_TRY(emu_unpermute(p, p->tc_Bd, d_B, s));
    if (d_M) API_TRY(emu_unpermute(p, p->tc_Md, d_M, s));
  } else if (p->tc_nsl) {
    if (d_B) API_TRY(tc_unpermute(p, p->tc_B, d_B, s));
    if (d_M) API_TRY(tc_unpermute(p, p->tc_M, d_M, s));
  } else {
    if (d_B) API_TRY(launch_unpermute(p, p->B, d_B, s));
    if (d_M) API_TRY(launch_unpermute(p, p->M, d_M, s));
  }
  return YGS_OK;
}

ygs_status ygs_get_weights(ygs_plan* p, int which, int patch, double* h_out) {
  if (!p || !h_out) return fail(YGS_ERR_INVALID_ARG, "NULL argument");
  if (which != 0 && which != 1) return fail(YGS_ERR_INVALID_ARG, "which must be 0 (U) or 1 (Q)");
  if (patch < 0 || patch >= p->n_patch) return fail(YGS_ERR_INVALID_ARG, "bad patch index");
  DeviceGuard guard(p->device);
  int g = p->symmetric ? 0 : patch;
  long long rows = p->nang[patch];
  std::vector<double> tmp((size_t)rows * p->K);
  const double* src = (which == 0 ? p->U : p->Q) + (size_t)p->pt.ang_off[g] * p->K;
  API_TRY(cudaMemcpy(tmp.data(), src, tmp.size() * sizeof(double), cudaMemcpyDeviceToHost));
  for (long long a = 0; a < rows; ++a)
    for (int ci = 0; ci < p->K; ++ci) {
      int c = p->col_perm[ci];
      double v = tmp[(size_t)a * p->K + ci];
      if (p->symmetric && patch == 1) {
        int l = 0;
        while ((l + 1) * (l + 1) <= c) ++l;
        if (((c - l * l + 1) / 2) & 1) v = -v;
      }
      h_out[(size_t)a * p->K + c] = v;
    }
  return YGS_OK;
}

ygs_status ygs_set_profiling(ygs_plan* p, int enable) {
  if (!p) return fail(YGS_ERR_INVALID_ARG, "plan is NULL");
  p->profiling = enable != 0;
  return YGS_OK;
}

ygs_status ygs_read_phase_times(ygs_plan* p, double* ms, int* n_calls) {
  if (!p || !ms || !n_calls) return fail(YGS_ERR_INVALID_ARG, "NULL argument");
  DeviceGuard guard(p->device);
  for (int k = 0; k < kPhases; ++k) ms[k] = 0.0;
  for (int c = 0; c < p->prof_used; ++c) {
    cudaEvent_t* ev = &p->prof_events[(size_t)c * (kPhases + 1)];
    API_TRY(cudaEventSynchronize(ev[kPhases]));
    for (int k = 0; k < kPhases; ++k) {
      float t = 0.f;
      API_TRY(cudaEventElapsedTime(&t, ev[k], ev[k + 1]));
      ms[k] += t;
    }
  }
  *n_calls = p->prof_used;
  p->prof_used = 0;
  return YGS_OK;
}

ygs_status ygs_debug_wait_timeout(ygs_plan* p, int spins, void* stream) {
  if (!p || spins < 1) return fail(YGS_ERR_INVALID_ARG, "bad arguments");
  DeviceGuard guard(p->device);
  cudaStream_t s = (cudaStream_t)stream;
  p->last_stream = s;
  API_TRY(debug_wait_timeout(p, spins, s));
  return YGS_OK;
}

int ygs_launches_per_solve(const ygs_plan* p) {
  return p ? (p->tc_nsl ? ((p->tc_fp16 || p->tc_emu) ? 5 : 4) : (p->precision == YGS_FP32 ? 5 : 3)) : 0;
}

ygs_status ygs_get_status(ygs_plan* p) {
  if (!p) return fail(YGS_ERR_INVALID_ARG, "plan is NULL");
  DeviceGuard guard(p->device);
  API_TRY(cudaStreamSynchronize(p->last_stream));
  int err = 0;
  API_TRY(cudaMemcpy(&err, p->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  API_TRY(cudaMemset(p->d_err, 0, sizeof(int)));
  // checked builds: the first out-of-range index any kernel on this device met
  int site = 0;
  long long index = 0;
  for (auto rd : {bounds_read_tc, bounds_read_fp64, bounds_read_emu}) {
    int s1 = 0;
    long long i1 = 0;
    API_TRY(rd(&s1, &i1));
    if (s1 && !site) {
      site = s1;
      index = i1;
    }
  }
  if (err) return fail((ygs_status)err, "device-side error word was set");
  if (site)
    return fail(YGS_ERR_BOUNDS, std::string("index ") + std::to_string(index) + " out of range at " +
                                    bounds_site_name(site));
  return YGS_OK;
}

int ygs_checked_build(void) { return YGS_DEBUG_BOUNDS; }

ygs_status ygs_debug_set_field_extent(ygs_plan* p, long long n) {
  if (!p || n < 0 || n > p->n_cells) return fail(YGS_ERR_INVALID_ARG, "bad arguments");
  if (!YGS_DEBUG_BOUNDS) return fail(YGS_ERR_UNSUPPORTED, "not a checked build");
  p->pt.n_cells = n;
  return YGS_OK;
}

}  // extern "C"
