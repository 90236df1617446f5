// Host <-> device layout: links from the MILC forward-only AoS order into the
// parity-split structure of arrays [parity][mu][elem][Vh] (FP64 and FP32
// copies, phases folded), and colour vectors between host parity order
// [Vh][3] and device [3][Vh]. The paper's own layout is an x86 AoSoA with
// 8-way links (Sec. 3); on the GPU a site-index-fastest SoA gives coalesced
// warp loads instead.
#include <cmath>
#include <complex>
#include <vector>

#include "sqcg_internal.cuh"

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ void coords_of(const Geom& g, long n, int& x, int& y, int& z, int& t) {
  x = (int)(n % g.Lx);
  n /= g.Lx;
  y = (int)(n % g.Ly);
  n /= g.Ly;
  z = (int)(n % g.Lz);
  t = (int)(n / g.Lz);
}

// one thread per (mu, site): raw[n][mu][9] -> out64[par][mu][e][n/2] (e < 9) and
// out32[par][mu][e][n/2] (e < nelem32: 9, or 6 for the 12-real form)
__global__ void k_pack_links(const double2* __restrict__ raw, Geom g, int fold, int hop, int nelem32,
                             double2* __restrict__ out64, float2* __restrict__ out32) {
  const long V = 2L * g.Vh;
  const long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= 4 * V) return;
  const int mu = (int)(tid / V);
  const long n = tid % V;
  int x, y, z, t;
  coords_of(g, n, x, y, z, t);
  const int par = (x + y + z + t) & 1;
  const long ih = n >> 1;
  double f = 1.0;
  if (fold) {
    int e = 0;
    if (mu == 1) e = x;
    if (mu == 2) e = x + y;
    if (mu == 3) e = x + y + z;
    if (e & 1) f = -f;
    if (mu == 3 && g.apbc && t + hop >= g.Lt) f = -f;
  }
  const double2* src = raw + (n * 4 + mu) * 9;
  const size_t base64 = ((size_t)par * 4 + mu) * 9 * g.Vh;
  const size_t base32 = ((size_t)par * 4 + mu) * nelem32 * g.Vh;
  for (int e = 0; e < 9; ++e) {
    const double2 u = src[e];
    const double2 v = make_double2(f * u.x, f * u.y);
    out64[base64 + (size_t)e * g.Vh + ih] = v;
    if (e < nelem32)
      out32[base32 + (size_t)e * g.Vh + ih] = make_float2(__double2float_rn(v.x), __double2float_rn(v.y));
  }
}

// host parity order [Vh][3] complex double -> device [3][Vh] (FP64 or FP32)
template <typename O2>
__global__ void k_aos_to_soa(const double2* __restrict__ aos, O2* __restrict__ soa, int Vh) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Vh) return;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const double2 v = aos[(size_t)i * 3 + c];
    O2 o;
    o.x = v.x;
    o.y = v.y;
    soa[(size_t)c * Vh + i] = o;
  }
}

// host parity order [Vh][3] complex double -> device [3][Vh] float-float (hi = fl32(v), lo = fl32(v - hi))
__global__ void k_aos_to_soa_ff(const double2* __restrict__ aos, float4* __restrict__ soa, int Vh) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Vh) return;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const double2 v = aos[(size_t)i * 3 + c];
    const float rh = __double2float_rn(v.x), ih = __double2float_rn(v.y);
    soa[(size_t)c * Vh + i] =
        make_float4(rh, __double2float_rn(v.x - (double)rh), ih, __double2float_rn(v.y - (double)ih));
  }
}

__global__ void k_soa_ff_to_aos(const float4* __restrict__ soa, double2* __restrict__ aos, int Vh) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Vh) return;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float4 v = soa[(size_t)c * Vh + i];
    aos[(size_t)i * 3 + c] = make_double2((double)v.x + (double)v.y, (double)v.z + (double)v.w);
  }
}

template <typename I2>
__global__ void k_soa_to_aos(const I2* __restrict__ soa, double2* __restrict__ aos, int Vh) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Vh) return;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const I2 v = soa[(size_t)c * Vh + i];
    aos[(size_t)i * 3 + c] = make_double2((double)v.x, (double)v.y);
  }
}

template <typename I2, typename O2>
__global__ void k_convert(const I2* __restrict__ in, O2* __restrict__ out, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const I2 v = in[i];
  O2 o;
  o.x = v.x;
  o.y = v.y;
  out[i] = o;
}

// 8-way FP32 backward links: out[p][mu][e][n_h] = -(U_mu(n - d mu))^dagger, from the
// folded FP64 forward links; e < nelem (6: first two rows for the 12-real form)
__global__ void k_pack_backward(const double2* __restrict__ fwd64, Geom g, int d, int nelem, float2* __restrict__ out) {
  const long V = 2L * g.Vh;
  const long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= 4 * V) return;
  const int mu = (int)(tid / V);
  const long n = tid % V;
  int c[4];
  long m = n;
  c[0] = (int)(m % g.Lx); m /= g.Lx;
  c[1] = (int)(m % g.Ly); m /= g.Ly;
  c[2] = (int)(m % g.Lz);
  c[3] = (int)(m / g.Lz);
  const int par = (c[0] + c[1] + c[2] + c[3]) & 1;
  const int Ls[4] = {g.Lx, g.Ly, g.Lz, g.Lt};
  int cb[4] = {c[0], c[1], c[2], c[3]};
  cb[mu] = ((c[mu] - d) % Ls[mu] + Ls[mu]) % Ls[mu];
  const long nb = cb[0] + (long)g.Lx * (cb[1] + (long)g.Ly * (cb[2] + (long)g.Lz * cb[3]));
  const int q = 1 - par;
  const size_t src = ((size_t)q * 4 + mu) * 9 * g.Vh + (nb >> 1);
  const size_t dst = ((size_t)par * 4 + mu) * nelem * g.Vh + (n >> 1);
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      const int e = a * 3 + b;
      if (e >= nelem) continue;
      const double2 u = fwd64[src + (size_t)(b * 3 + a) * g.Vh];  // element (b, a) of the forward link
      out[dst + (size_t)e * g.Vh] = make_float2(__double2float_rn(-u.x), __double2float_rn(u.y));
    }
}

typedef std::complex<double> cd;

// 12-real eligibility: every long link is s * W, W in SU(3), |s| global.
// With the phases folded by the caller, s carries eta_mu(n) and the boundary
// sign; they are divided out before the scale is compared.
bool recon_check(const sqcg_ctx* ctx, const double* lng, double* s0_out) {
  const int* L = ctx->L;
  const long V = (long)L[0] * L[1] * L[2] * L[3];
  const bool folded = (ctx->flags & SQCG_PHASES_FOLDED) != 0;
  double s0 = 0.0;
  for (long n = 0; n < V; ++n) {
    long m = n;
    const int x = (int)(m % L[0]); m /= L[0];
    const int y = (int)(m % L[1]); m /= L[1];
    const int z = (int)(m % L[2]);
    const int t = (int)(m / L[2]);
    for (int mu = 0; mu < 4; ++mu) {
      const double* p = lng + ((size_t)n * 4 + mu) * 18;
      cd U[3][3];
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) U[a][b] = cd(p[(a * 3 + b) * 2], p[(a * 3 + b) * 2 + 1]);
      const cd det = U[0][0] * (U[1][1] * U[2][2] - U[1][2] * U[2][1]) -
                     U[0][1] * (U[1][0] * U[2][2] - U[1][2] * U[2][0]) +
                     U[0][2] * (U[1][0] * U[2][1] - U[1][1] * U[2][0]);
      const double s = std::cbrt(det.real());
      if (!(std::fabs(s) > 0.0) || !std::isfinite(s)) return false;
      const double s3 = std::fabs(s * s * s);
      if (std::abs(det.imag()) > 1e-12 * s3) return false;
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
          cd uu = 0;
          for (int c = 0; c < 3; ++c) uu += U[a][c] * std::conj(U[b][c]);
          if (a == b) uu -= s * s;
          if (std::abs(uu) > 1e-12 * s * s) return false;
        }
      double f = 1.0;
      if (folded) {
        int e = 0;
        if (mu == 1) e = x;
        if (mu == 2) e = x + y;
        if (mu == 3) e = x + y + z;
        if (e & 1) f = -f;
        if (mu == 3 && (ctx->flags & SQCG_ANTIPERIODIC_T) && t + 3 >= L[3]) f = -f;
      }
      const double s_unfolded = s * f;
      if (n == 0 && mu == 0) s0 = s_unfolded;
      else if (std::fabs(s_unfolded - s0) > 1e-12 * std::fabs(s0)) return false;
    }
  }
  *s0_out = s0;
  return true;
}

int ensure_stage(sqcg_ctx* ctx, size_t bytes) {
  if (ctx->stage_bytes >= bytes) return SQCG_OK;
  if (ctx->stage) cudaFree(ctx->stage);
  ctx->stage = nullptr;
  ctx->stage_bytes = 0;
  if (cudaMalloc(&ctx->stage, bytes) != cudaSuccess) {
    cudaGetLastError();
    return SQCG_ERR_NO_MEMORY;
  }
  ctx->stage_bytes = bytes;
  return SQCG_OK;
}

}  // namespace

namespace {

// fat, lng: host order [V][4][3][3] complex, in host memory or (on_device) in device memory
int load_links(sqcg_ctx* ctx, const double* fat, const double* lng, int opts, bool on_device) {
  if (!fat || !lng) return SQCG_ERR_INVALID_ARG;
  if (opts & ~(SQCG_RECON12_LONG | SQCG_EIGHT_WAY)) return SQCG_ERR_INVALID_ARG;
  const bool recon = (opts & SQCG_RECON12_LONG) != 0;
  const bool eightway = (opts & SQCG_EIGHT_WAY) != 0;
  double s0 = 1.0;
  if (recon) {
    if (on_device) {  // the eligibility test runs on the host
      std::vector<double> h((size_t)2 * ctx->g.Vh * 4 * 18);
      SQCG_CUDA_TRY(cudaMemcpy(h.data(), lng, h.size() * sizeof(double), cudaMemcpyDeviceToHost));
      if (!recon_check(ctx, h.data(), &s0)) return SQCG_ERR_RECON_REJECTED;
    } else if (!recon_check(ctx, lng, &s0)) {
      return SQCG_ERR_RECON_REJECTED;
    }
  }

  const size_t Vh = ctx->g.Vh, V = 2 * Vh;
  // the 12-real form is used for the FP32 copy only: on this GPU the FP64 Dslash is
  // bound by FP64 arithmetic, which rebuilding the third row would only add to
  const int nl32 = recon ? 6 : 9;
  const size_t nfat = 2 * 4 * 9 * Vh, nlng64 = 2 * 4 * 9 * Vh, nlng32 = 2 * 4 * (size_t)nl32 * Vh;
  cudaStream_t s = ctx->stream;

  // drop earlier links
  SQCG_CUDA_TRY(cudaStreamSynchronize(s));
  cudaFree(ctx->fat64); cudaFree(ctx->lng64); cudaFree(ctx->fat32); cudaFree(ctx->lng32);
  cudaFree(ctx->fatb32); cudaFree(ctx->lngb32);
  cudaFree(ctx->fatff); cudaFree(ctx->lngff);
  ctx->fat64 = ctx->lng64 = nullptr;
  ctx->fat32 = ctx->lng32 = nullptr;
  ctx->fatb32 = ctx->lngb32 = nullptr;
  ctx->fatff = ctx->lngff = nullptr;
  ctx->eightway = false;
  ctx->have_links = false;
  free_graphs(ctx);
  free_batch_plan(ctx);

  void* raw = nullptr;
  bool ok = cudaMalloc((void**)&ctx->fat64, nfat * sizeof(double2)) == cudaSuccess &&
            cudaMalloc((void**)&ctx->lng64, nlng64 * sizeof(double2)) == cudaSuccess &&
            cudaMalloc((void**)&ctx->fat32, nfat * sizeof(float2)) == cudaSuccess &&
            cudaMalloc((void**)&ctx->lng32, nlng32 * sizeof(float2)) == cudaSuccess &&
            cudaMalloc((void**)&ctx->fatff, nfat * sizeof(float4)) == cudaSuccess &&
            cudaMalloc((void**)&ctx->lngff, nlng64 * sizeof(float4)) == cudaSuccess &&
            (on_device || cudaMalloc(&raw, V * 4 * 9 * sizeof(double2)) == cudaSuccess);
  if (!ok) {
    cudaGetLastError();
    cudaFree(raw);
    cudaFree(ctx->fat64); cudaFree(ctx->lng64); cudaFree(ctx->fat32); cudaFree(ctx->lng32);
    cudaFree(ctx->fatff); cudaFree(ctx->lngff);
    ctx->fat64 = ctx->lng64 = nullptr;
    ctx->fat32 = ctx->lng32 = nullptr;
    ctx->fatff = ctx->lngff = nullptr;
    return SQCG_ERR_NO_MEMORY;
  }
  const int fold = (ctx->flags & SQCG_PHASES_FOLDED) ? 0 : 1;
  const long nthreads = 4 * (long)V;
  const int grid = (int)((nthreads + kThreads - 1) / kThreads);
  int rc = SQCG_OK;
  do {
    const double2* src = (const double2*)fat;
    if (!on_device) {
      if (cudaMemcpyAsync(raw, fat, V * 4 * 9 * sizeof(double2), cudaMemcpyHostToDevice, s) != cudaSuccess) { rc = SQCG_ERR_CUDA; break; }
      src = (const double2*)raw;
    }
    k_pack_links<<<grid, kThreads, 0, s>>>(src, ctx->g, fold, 1, 9, ctx->fat64, ctx->fat32);
    if (cudaGetLastError() != cudaSuccess) { rc = SQCG_ERR_CUDA; break; }
    src = (const double2*)lng;
    if (!on_device) {
      // the fat pass must finish reading the staging buffer before it is overwritten (same stream)
      if (cudaMemcpyAsync(raw, lng, V * 4 * 9 * sizeof(double2), cudaMemcpyHostToDevice, s) != cudaSuccess) { rc = SQCG_ERR_CUDA; break; }
      src = (const double2*)raw;
    }
    k_pack_links<<<grid, kThreads, 0, s>>>(src, ctx->g, fold, 3, nl32, ctx->lng64, ctx->lng32);
    if (cudaGetLastError() != cudaSuccess) { rc = SQCG_ERR_CUDA; break; }
    // the float-float copy of the folded FP64 links (reliable-update arithmetic)
    if (launch_split_ff(ctx->fat64, ctx->fatff, nfat, s) != SQCG_OK) { rc = SQCG_ERR_CUDA; break; }
    if (launch_split_ff(ctx->lng64, ctx->lngff, nlng64, s) != SQCG_OK) { rc = SQCG_ERR_CUDA; break; }
    if (cudaStreamSynchronize(s) != cudaSuccess) { rc = SQCG_ERR_CUDA; break; }
  } while (0);
  cudaFree(raw);
  if (rc == SQCG_OK && eightway) {
    if (cudaMalloc((void**)&ctx->fatb32, nfat * sizeof(float2)) != cudaSuccess ||
        cudaMalloc((void**)&ctx->lngb32, nlng32 * sizeof(float2)) != cudaSuccess) {
      cudaGetLastError();
      cudaFree(ctx->fatb32); cudaFree(ctx->lngb32);
      ctx->fatb32 = ctx->lngb32 = nullptr;
      return SQCG_ERR_NO_MEMORY;
    }
    k_pack_backward<<<grid, kThreads, 0, s>>>(ctx->fat64, ctx->g, 1, 9, ctx->fatb32);
    k_pack_backward<<<grid, kThreads, 0, s>>>(ctx->lng64, ctx->g, 3, nl32, ctx->lngb32);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) rc = SQCG_ERR_CUDA;
  }
  if (rc != SQCG_OK) {
    sqcg_set_last_cuda_error(cudaGetLastError(), "load_links", __FILE__, __LINE__);
    return rc;
  }
  ctx->eightway = eightway;
  ctx->recon = recon;
  ctx->long_scale = s0;
  ctx->have_links = true;
  static unsigned long long generation = 0;
  ctx->links_gen = __atomic_add_fetch(&generation, 1ULL, __ATOMIC_RELAXED);
  return SQCG_OK;
}

}  // namespace

int layout_load_links(sqcg_ctx* ctx, const double* fat, const double* lng, int opts) {
  return load_links(ctx, fat, lng, opts, false);
}

int layout_load_links_device(sqcg_ctx* ctx, const double* fat, const double* lng, int opts) {
  return load_links(ctx, fat, lng, opts, true);
}

int layout_pack_spinor(sqcg_ctx* ctx, int prec, const double* host, void* dev) {
  if (!host || !dev || (prec != SQCG_F64 && prec != SQCG_F32 && prec != SQCG_FF)) return SQCG_ERR_INVALID_ARG;
  const int Vh = ctx->g.Vh;
  const size_t bytes = (size_t)Vh * 3 * sizeof(double2);
  SQCG_TRY(ensure_stage(ctx, bytes));
  cudaStream_t s = ctx->stream;
  SQCG_CUDA_TRY(cudaMemcpyAsync(ctx->stage, host, bytes, cudaMemcpyHostToDevice, s));
  if (prec == SQCG_F64)
    k_aos_to_soa<double2><<<grid_for(Vh, kThreads), kThreads, 0, s>>>((const double2*)ctx->stage, (double2*)dev, Vh);
  else if (prec == SQCG_FF)
    k_aos_to_soa_ff<<<grid_for(Vh, kThreads), kThreads, 0, s>>>((const double2*)ctx->stage, (float4*)dev, Vh);
  else
    k_aos_to_soa<float2><<<grid_for(Vh, kThreads), kThreads, 0, s>>>((const double2*)ctx->stage, (float2*)dev, Vh);
  SQCG_CUDA_TRY(cudaGetLastError());
  return SQCG_OK;
}

int layout_unpack_spinor(sqcg_ctx* ctx, int prec, const void* dev, double* host) {
  if (!host || !dev || (prec != SQCG_F64 && prec != SQCG_F32 && prec != SQCG_FF)) return SQCG_ERR_INVALID_ARG;
  const int Vh = ctx->g.Vh;
  const size_t bytes = (size_t)Vh * 3 * sizeof(double2);
  SQCG_TRY(ensure_stage(ctx, bytes));
  cudaStream_t s = ctx->stream;
  if (prec == SQCG_F64)
    k_soa_to_aos<double2><<<grid_for(Vh, kThreads), kThreads, 0, s>>>((const double2*)dev, (double2*)ctx->stage, Vh);
  else if (prec == SQCG_FF)
    k_soa_ff_to_aos<<<grid_for(Vh, kThreads), kThreads, 0, s>>>((const float4*)dev, (double2*)ctx->stage, Vh);
  else
    k_soa_to_aos<float2><<<grid_for(Vh, kThreads), kThreads, 0, s>>>((const float2*)dev, (double2*)ctx->stage, Vh);
  SQCG_CUDA_TRY(cudaGetLastError());
  SQCG_CUDA_TRY(cudaMemcpyAsync(host, ctx->stage, bytes, cudaMemcpyDeviceToHost, s));
  SQCG_CUDA_TRY(cudaStreamSynchronize(s));
  return SQCG_OK;
}

int layout_convert(sqcg_ctx* ctx, int from_prec, const void* src, int to_prec, void* dst, cudaStream_t s) {
  const int n = ctx->g.Vh * 3;
  const int grid = grid_for(n, kThreads);
  if (from_prec == SQCG_F64 && to_prec == SQCG_F32)
    k_convert<double2, float2><<<grid, kThreads, 0, s>>>((const double2*)src, (float2*)dst, n);
  else if (from_prec == SQCG_F32 && to_prec == SQCG_F64)
    k_convert<float2, double2><<<grid, kThreads, 0, s>>>((const float2*)src, (double2*)dst, n);
  else if (from_prec == to_prec)
    SQCG_CUDA_TRY(cudaMemcpyAsync(dst, src, (size_t)n * (from_prec == SQCG_F64 ? 16 : 8), cudaMemcpyDeviceToDevice, s));
  else
    return SQCG_ERR_INVALID_ARG;
  SQCG_CUDA_TRY(cudaGetLastError());
  return SQCG_OK;
}

unsigned long long sqcg_links_generation(const sqcg_ctx* ctx) { return ctx->links_gen; }
