// adept_build_tables_noalloc: the physics-table build for callers that cannot allocate
// device memory. Same closed forms and quadrature as adept_build_tables, fused into one
// kernel (one block per material) whose working rows live in a file-scope __device__
// array instead of a caller-provided arena.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/adept.h"
#include "device.cuh"
#include "layout.h"
#include "physics_init.cuh"

namespace adept {
namespace {

constexpr int kRows = 17;  // 14 value rows + 3 rows of per-bin range integrals
constexpr int kNoAllocMat = ADEPT_NOALLOC_MAX_MATERIALS;

// Working rows of every call, on every device that loads the library (held until exit):
// kNoAllocMat x 17 x 289 doubles = 157 KB. Calls share it; each call writes every word it
// reads before reading it, so nothing needs clearing, but calls that overlap on the GPU
// race on it.
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocMat * kRows * kNNode];

struct MatIn {
  double v[kNoAllocMat][kMatRec];  // material records (elements only), passed by value
};

enum { R_MUC, R_MUP, R_MUPH, R_SFULL, R_SE, R_IE, R_BE, R_SP, R_IP, R_BP, R_AP, R_RFULL, R_RE, R_RP, R_BFULL, R_BE_, R_BP_ };

// one block per material; output tables [m][12][289] (gamma 3, e- 4, e+ 5) and cuts [m][2]
__global__ void k_tables_noalloc(MatIn in, double range_cut, double* scratch, double* out, double* cuts) {
  const int m = blockIdx.x;
  __shared__ MatDev M;
  __shared__ double tc, kc;
  if (threadIdx.x == 0) init::setup_material(in.v[m], &M);
  __syncthreads();
  double* w = scratch + (size_t)m * kRows * kNNode;
  double* o = out + (size_t)m * 12 * kNNode;
  const int i = threadIdx.x;
  if (M.vacuum) {
    for (int k = i; k < 12 * kNNode; k += blockDim.x) o[k] = 0.0;
    if (i == 0) { cuts[2 * m] = 0.0; cuts[2 * m + 1] = 0.0; }
    return;
  }
  auto full = [&](double T) { return init::dedx_col(M, T, T, false) + init::dedx_rad(M, T, T); };
  if (i < kNNode) {
    const double E = init::node_E(i);
    w[R_MUC * kNNode + i] = init::mu_compton(M, E);
    w[R_MUP * kNNode + i] = init::mu_pair(M, E);
    w[R_MUPH * kNNode + i] = init::mu_photo(M, E);
    w[R_SFULL * kNNode + i] = full(E);
    if (i < kNNode - 1) w[R_BFULL * kNNode + i] = init::bin_integral(i, full);
  }
  __syncthreads();
  if (i == 0) {
    init::prefix_range(w + R_SFULL * kNNode, w + R_BFULL * kNNode, w + R_RFULL * kNNode);
    auto mu = [&](int k) { return w[R_MUC * kNNode + k] + w[R_MUP * kNNode + k] + w[R_MUPH * kNNode + k]; };
    tc = init::clamp_cut(init::range_threshold(w + R_RFULL * kNNode, range_cut));
    kc = init::clamp_cut(init::gamma_threshold(mu, range_cut));
    cuts[2 * m] = tc;
    cuts[2 * m + 1] = kc;
  }
  __syncthreads();
  const double Tc = tc, Kc = kc;
  auto se = [&](double T) { return init::dedx_col(M, T, Tc, false) + init::dedx_rad(M, T, Kc); };
  auto sp = [&](double T) { return init::dedx_col(M, T, Tc, true) + init::dedx_rad(M, T, Kc); };
  if (i < kNNode) {
    const double T = init::node_E(i);
    w[R_SE * kNNode + i] = se(T);
    w[R_IE * kNNode + i] = init::lambda_ioni(M, T, Tc, false);
    w[R_BE * kNNode + i] = init::lambda_brem(M, T, Kc);
    w[R_SP * kNNode + i] = sp(T);
    w[R_IP * kNNode + i] = init::lambda_ioni(M, T, Tc, true);
    w[R_BP * kNNode + i] = init::lambda_brem(M, T, Kc);
    w[R_AP * kNNode + i] = init::lambda_annih(M, T);
    if (i < kNNode - 1) {
      w[R_BE_ * kNNode + i] = init::bin_integral(i, se);
      w[R_BP_ * kNNode + i] = init::bin_integral(i, sp);
    }
  }
  __syncthreads();
  if (i == 0) init::prefix_range(w + R_SE * kNNode, w + R_BE_ * kNNode, w + R_RE * kNNode);
  if (i == 1) init::prefix_range(w + R_SP * kNNode, w + R_BP_ * kNNode, w + R_RP * kNNode);
  __syncthreads();
  const int rows[12] = {R_MUC, R_MUP, R_MUPH, R_SE, R_RE, R_IE, R_BE, R_SP, R_RP, R_IP, R_BP, R_AP};
  if (i < kNNode)
    for (int r = 0; r < 12; ++r) o[r * kNNode + i] = w[rows[r] * kNNode + i];
}

std::mutex g_mu;
double* g_ptr[256] = {};

}  // namespace
}  // namespace adept

using namespace adept;

extern "C" int adept_build_tables_noalloc(const adept_material* materials, int32_t n_materials, double range_cut_mm,
                                          double* dev_tables, double* dev_cuts, void* stream) {
  if (!materials || !dev_tables || !dev_cuts) return ADEPT_EINVAL;
  if (n_materials < 1 || n_materials > kNoAllocMat) return ADEPT_EINVAL;  // beyond the static scratch
  if (!(range_cut_mm > 0.0)) return ADEPT_EINVAL;
  MatIn in{};
  for (int m = 0; m < n_materials; ++m) {
    const adept_material& t = materials[m];
    if (t.n_elements != 0) return ADEPT_EINVAL;  // single elements only
    if (t.Z < 0 || t.Z > 100 || (t.Z > 0 && !(t.A_g_mol > 0 && t.density_g_cm3 > 0 && t.I_eV > 0))) return ADEPT_EINVAL;
    in.v[m][0] = t.Z; in.v[m][1] = t.A_g_mol; in.v[m][2] = t.density_g_cm3; in.v[m][3] = t.I_eV; in.v[m][4] = 0.0;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return ADEPT_ECUDA;
  double* scratch;
  {
    // the array's device address, once per device with that device current; host code
    // cannot use the symbol itself (it names a host-side stand-in)
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_ptr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return ADEPT_ECUDA;
      g_ptr[dev] = static_cast<double*>(p);
    }
    scratch = g_ptr[dev];
  }
  k_tables_noalloc<<<n_materials, 320, 0, static_cast<cudaStream_t>(stream)>>>(in, range_cut_mm, scratch, dev_tables,
                                                                               dev_cuts);
  return cudaGetLastError() == cudaSuccess ? ADEPT_OK : ADEPT_ECUDA;
}
