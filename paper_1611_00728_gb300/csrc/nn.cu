// Learned gauge-covariant preconditioner and flexible CG.
//
// The paper has no preconditioner; this is the learned preconditioner of a
// flexible CG around its single-mass CG (Sec. 3). Network N (1,472
// parameters): three parallel-transport convolution layers over the fat links
// (channels 1 -> 8 -> 8 -> 1, 9 taps: self + 8 one-hop neighbours, complex
// colour-blind weights stored in BF16, FP32 accumulation), a gauge-invariant
// gate h <- h sigmoid(a |h|^2 + b) after layers 1 and 2, input scaled to unit
// RMS and output scaled back (N(c r) = c N(r)). Gauge covariance is exact:
// weights mix channels only, links carry colour, gates see only |h|.
//
// Training minimises L = <d, A d> / <e, r>, d = N(r) - e, over (residual,
// error) pairs produced by plain CG: the A-norm of the preconditioned error
// relative to that of e (or, selectable, the A^2-norm <A d, A d> / <r, r>,
// the residual of the preconditioned step). dL/dz (2 A d / <e, r>, or
// 2 A A d / <r, r>) is back-propagated with
// hand-written kernels (adjoint convolutions, gate backward, weight-gradient
// reductions) and the weights follow Adam (FP32 master, BF16 forward copy).
//
// Flexible CG (Notay's FCG with one stored direction, Polak-Ribiere beta):
//   q = A p; alpha = <z,r>/<p,q>; x += alpha p; r_old = r; r -= alpha q;
//   z = N(r); beta = (<z,r> - <z,r_old>) / <z_old,r_old>; p = z + beta p,
// with FP32 vectors, FP64 x and reliable updates as in the mixed CG, run as
// one CUDA graph (WHILE node; SQCG_LAUNCH_MODE=eager launches the same kernels
// one at a time). On breakdown or no convergence it falls back to the
// mixed-precision CG from the current iterate.
#include <chrono>
#include <cuda_bf16.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "solver_device.cuh"
#include "sqcg_internal.cuh"

namespace {

constexpr int NT = 9;   // taps: 0 self, 1 + 2 mu forward hop, 2 + 2 mu backward hop
constexpr int CH = 8;   // hidden channels
constexpr int OFF_W1 = 0;                          // [9][8][1] complex
constexpr int OFF_W2 = OFF_W1 + NT * CH * 1 * 2;   // [9][8][8] complex
constexpr int OFF_W3 = OFF_W2 + NT * CH * CH * 2;  // [9][1][8] complex
constexpr int OFF_G = OFF_W3 + NT * 1 * CH * 2;    // gate a1[8], b1[8], a2[8], b2[8]
constexpr int NPARAM = OFF_G + 4 * CH;             // 1472
constexpr int NWEIGHT = OFF_G / 2;                 // complex weights: 720
constexpr int kThreads = 128;
constexpr int kRedThreads = 256;

static_assert(NPARAM == 1472, "parameter layout");

// ---------------------------------------------------------------------------
// geometry helpers (same site numbering as the Dslash)
// ---------------------------------------------------------------------------
struct Site {
  int i, par, x, y, z, t, row;
};

__device__ __forceinline__ Site site_of(const Geom& g, int i, int par) {
  Site s;
  s.i = i;
  s.par = par;
  const int xh = i % g.Lxh;
  int r = i / g.Lxh;
  s.y = r % g.Ly;
  r /= g.Ly;
  s.z = r % g.Lz;
  s.t = r / g.Lz;
  s.x = 2 * xh + ((s.y + s.z + s.t + par) & 1);
  s.row = i - xh;
  return s;
}

// half-lattice index of the neighbour n + d mu (d = +1 or -1); it has the other parity
__device__ __forceinline__ int nbr(const Geom& g, const Site& s, int mu, int d) {
  if (mu == 0) {
    int xp = s.x + d;
    if (xp >= g.Lx) xp -= g.Lx;
    if (xp < 0) xp += g.Lx;
    return s.row + (xp >> 1);
  }
  const int c = (mu == 1) ? s.y : (mu == 2) ? s.z : s.t;
  const int L = (mu == 1) ? g.Ly : (mu == 2) ? g.Lz : g.Lt;
  const int st = (mu == 1) ? g.sy : (mu == 2) ? g.sz : g.st;
  int j = s.i + d * st;
  if (c + d >= L) j -= L * st;
  if (c + d < 0) j += L * st;
  return j;
}

__device__ __forceinline__ void cmac(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(a.y, b.x, acc.y);
}

// (a.x b.x + c.x, a.y b.y + c.y) as one packed two-lane FP32 FMA (sm_100 and later); each
// lane is an ordinary round-to-nearest FMA, so the results equal two fmaf calls
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\tmov.b64 rc, {%6, %7};\n\t"
      "fma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return d;
}

__device__ __forceinline__ void load_link9(const float2* __restrict__ U, int Vh, int idx, float2 (&u)[9]) {
#pragma unroll
  for (int e = 0; e < 9; ++e) u[e] = __ldg(U + (size_t)e * Vh + idx);
}

// U v (dag = false) or U^dag v (dag = true) for a link already in registers
__device__ __forceinline__ void apply_link(const float2 (&u)[9], bool dag, const float2 (&v)[3], float2 (&out)[3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      if (!dag) {
        cmac(acc, u[a * 3 + b], v[b]);
      } else {
        const float2 c = make_float2(u[b * 3 + a].x, -u[b * 3 + a].y);
        cmac(acc, c, v[b]);
      }
    }
    out[a] = acc;
  }
}

// ---------------------------------------------------------------------------
// convolution layer
// ---------------------------------------------------------------------------
enum InMode { IN_FULL = 0, IN_EVEN_SCALED = 1 };
enum OutMode { OUT_FULL = 0, OUT_GATE_TRAIN = 1, OUT_GATE_INFER = 2, OUT_EVEN_SCALED = 3 };

struct ConvArgs {
  Geom g;
  const float2* fat[2];   // FP32 fat links of each parity, [mu][9][Vh]
  const float2* in;       // IN_FULL: [CIN][2][3][Vh]; IN_EVEN_SCALED: even vector [3][Vh]
  float2* out;            // OUT_FULL / OUT_GATE_*: [COUT][2][3][Vh]; OUT_EVEN_SCALED: even vector [3][Vh]
  float2* pre;            // OUT_GATE_TRAIN: pre-activations [COUT][2][3][Vh]
  const float2* W;        // [9][COUT][CIN] complex (FP32 copy of BF16 values)
  const float* gate_a;    // [COUT]
  const float* gate_b;
  const double* scale;    // IN_EVEN_SCALED: input scale; OUT_EVEN_SCALED: output scale
  const SolverState* st;  // gate (may be null)
  int gate;
  int par0;               // first output parity handled (threads cover npar parities)
  int npar;
};

// one lane per site: the layers with one input or one output channel (the 8 -> 8 layer is
// k_conv88 below)
template <int CIN, int COUT, int IN, int OUT>
__global__ void __launch_bounds__(kThreads, 4) k_conv(ConvArgs a) {
  if (a.st && !gate_open(a.st, a.gate)) return;
  __shared__ float2 W[NT * COUT * CIN];
  for (int j = threadIdx.x; j < NT * COUT * CIN; j += blockDim.x) W[j] = a.W[j];
  __syncthreads();
  const Geom& g = a.g;
  const int Vh = g.Vh;
  const int gid = blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= a.npar * Vh) return;
  const int par = a.par0 + gid / Vh;
  const int i = gid % Vh;
  const int q = 1 - par;
  const Site s = site_of(g, i, par);
  const float sc = (IN == IN_EVEN_SCALED) ? (float)*a.scale : 1.f;

  float2 acc[COUT][3];
#pragma unroll
  for (int o = 0; o < COUT; ++o)
#pragma unroll
    for (int c = 0; c < 3; ++c) acc[o][c] = make_float2(0.f, 0.f);

  // input channel ci at parity pp, half index j
  auto load_in = [&](int ci, int pp, int j, float2 (&v)[3]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      if (IN == IN_FULL) {
        v[c] = __ldg(a.in + (((size_t)ci * 2 + pp) * 3 + c) * Vh + j);
      } else {
        const float2 t = __ldg(a.in + (size_t)c * Vh + j);
        v[c] = make_float2(t.x * sc, t.y * sc);
      }
    }
  };
  auto mix = [&](int tap, const float2 (&t)[3], int ci) {
#pragma unroll
    for (int o = 0; o < COUT; ++o) {
      const float2 w = W[(tap * COUT + o) * CIN + ci];
#pragma unroll
      for (int c = 0; c < 3; ++c) cmac(acc[o][c], w, t[c]);
    }
  };

  // self tap (input of the same parity; an even-only input is zero on odd sites)
  if (IN == IN_FULL || par == 0) {
#pragma unroll
    for (int ci = 0; ci < CIN; ++ci) {
      float2 v[3];
      load_in(ci, par, i, v);
      mix(0, v, ci);
    }
  }
  // hops (input of the other parity); each link is loaded once and applied to every channel
  if (IN == IN_FULL || q == 0) {
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
#pragma unroll
      for (int dir = 0; dir < 2; ++dir) {
        const int j = nbr(g, s, mu, dir == 0 ? +1 : -1);
        float2 u[9];
        if (dir == 0) load_link9(a.fat[par] + (size_t)mu * 9 * Vh, Vh, i, u);  // F_mu(n)
        else load_link9(a.fat[q] + (size_t)mu * 9 * Vh, Vh, j, u);             // F_mu(n - mu)
        const int tap = 1 + 2 * mu + dir;
        if constexpr (COUT == 1 && CIN > 1) {
          // one output channel: the weights mix channels and the link acts on colour, so
          // sum_ci w_ci (U v_ci) = U (sum_ci w_ci v_ci): mix first, transport once
          float2 m[3] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
#pragma unroll 2
          for (int ci = 0; ci < CIN; ++ci) {
            float2 v[3];
            load_in(ci, q, j, v);
            const float2 w = W[tap * CIN + ci];
#pragma unroll
            for (int c = 0; c < 3; ++c) cmac(m[c], w, v[c]);
          }
          float2 t[3];
          apply_link(u, dir == 1, m, t);
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            acc[0][c].x += t[c].x;
            acc[0][c].y += t[c].y;
          }
        } else {
#pragma unroll 2
          for (int ci = 0; ci < CIN; ++ci) {
            float2 v[3], t[3];
            load_in(ci, q, j, v);
            apply_link(u, dir == 1, v, t);
            mix(tap, t, ci);
          }
        }
      }
    }
  }
  // epilogue
  if (OUT == OUT_EVEN_SCALED) {
    const float os = (float)*a.scale;
#pragma unroll
    for (int c = 0; c < 3; ++c) a.out[(size_t)c * Vh + i] = make_float2(acc[0][c].x * os, acc[0][c].y * os);
  } else {
#pragma unroll
    for (int o = 0; o < COUT; ++o) {
      float gf = 1.f;
      if (OUT == OUT_GATE_TRAIN || OUT == OUT_GATE_INFER) {
        float n2 = 0.f;
#pragma unroll
        for (int c = 0; c < 3; ++c) n2 = fmaf(acc[o][c].x, acc[o][c].x, fmaf(acc[o][c].y, acc[o][c].y, n2));
        gf = 1.f / (1.f + __expf(-(a.gate_a[o] * n2 + a.gate_b[o])));
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const size_t k = (((size_t)o * 2 + par) * 3 + c) * Vh + i;
        if (OUT == OUT_GATE_TRAIN) a.pre[k] = acc[o][c];
        a.out[k] = make_float2(acc[o][c].x * gf, acc[o][c].y * gf);
      }
    }
  }
}

// The 8 -> 8 layer with two lanes per site. Each lane accumulates 4 of the 8 output
// channels and transports 4 of the 8 input channels per hop; the two lanes swap their
// transported vectors with a warp shuffle, so no product is done twice and a lane holds half
// the accumulators of the one-lane form (more resident warps to hide the neighbour loads).
// Lanes past the end compute on a clamped site and store nothing, so every lane of a warp
// takes part in the shuffles.
template <int OUT>
__global__ void __launch_bounds__(kThreads, 5) k_conv88(ConvArgs a) {
  if (a.st && !gate_open(a.st, a.gate)) return;
  // weights as [tap][c_in][c_out], each complex w stored as (w.x, w.x, -w.y, w.y): the two packed
  // operands of acc += w t in two-lane FMAs, acc = (w.x, w.x) (t.x, t.y) + (-w.y, w.y) (t.y, t.x) + acc,
  // which rounds exactly as the scalar complex multiply-add (same products, same order per lane)
  __shared__ float4 W[NT * CH * CH];
  for (int j = threadIdx.x; j < NT * CH * CH; j += blockDim.x) {
    const int tap = j / (CH * CH), o = (j / CH) % CH, ci = j % CH;
    const float2 w = a.W[j];
    W[(tap * CH + ci) * CH + o] = make_float4(w.x, w.x, -w.y, w.y);
  }
  __syncthreads();
  const Geom& g = a.g;
  const int Vh = g.Vh;
  const int gid = blockIdx.x * blockDim.x + threadIdx.x;
  const int h = gid & 1;  // this lane's half of the channels
  const int site = gid >> 1;
  const bool valid = site < a.npar * Vh;
  const int sv = valid ? site : 0;
  const int par = a.par0 + sv / Vh;
  const int i = sv % Vh;
  const int q = 1 - par;
  const Site s = site_of(g, i, par);

  float2 acc[4][3];
#pragma unroll
  for (int o = 0; o < 4; ++o)
#pragma unroll
    for (int c = 0; c < 3; ++c) acc[o][c] = make_float2(0.f, 0.f);
  auto load_in = [&](int ci, int pp, int j, float2 (&v)[3]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) v[c] = __ldg(a.in + (((size_t)ci * 2 + pp) * 3 + c) * Vh + j);
  };
  auto mix1 = [&](int tap, int ci, const float2 (&t)[3]) {
    const float4* wq = W + (tap * CH + ci) * CH + 4 * h;
    float2 ts[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) ts[c] = make_float2(t[c].y, t[c].x);
#pragma unroll
    for (int o = 0; o < 4; ++o) {
      const float4 w = wq[o];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        acc[o][c] = ffma2(make_float2(w.x, w.y), t[c], acc[o][c]);
        acc[o][c] = ffma2(make_float2(w.z, w.w), ts[c], acc[o][c]);
      }
    }
  };
  // self tap: every input channel at the site (the partner lane reads the same values, from L1)
#pragma unroll 2
  for (int ci = 0; ci < CH; ++ci) {
    float2 v[3];
    load_in(ci, par, i, v);
    mix1(0, ci, v);
  }
  // hops
#pragma unroll 1
  for (int mu = 0; mu < 4; ++mu) {
#pragma unroll
    for (int dir = 0; dir < 2; ++dir) {
      const int j = nbr(g, s, mu, dir == 0 ? +1 : -1);
      const int tap = 1 + 2 * mu + dir;
      float2 t[4][3];
      {
        float2 u[9];
        if (dir == 0) load_link9(a.fat[par] + (size_t)mu * 9 * Vh, Vh, i, u);  // F_mu(n)
        else load_link9(a.fat[q] + (size_t)mu * 9 * Vh, Vh, j, u);             // F_mu(n - mu)
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          float2 v[3];
          load_in(4 * h + k, q, j, v);
          apply_link(u, dir == 1, v, t[k]);
        }
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        float2 pt[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          pt[c].x = __shfl_xor_sync(0xffffffffu, t[k][c].x, 1);
          pt[c].y = __shfl_xor_sync(0xffffffffu, t[k][c].y, 1);
        }
        mix1(tap, 4 * h + k, t[k]);
        mix1(tap, 4 * (1 - h) + k, pt);
      }
    }
  }
  if (!valid) return;
#pragma unroll
  for (int o4 = 0; o4 < 4; ++o4) {
    const int o = 4 * h + o4;
    float gf = 1.f;
    if (OUT == OUT_GATE_TRAIN || OUT == OUT_GATE_INFER) {
      float n2 = 0.f;
#pragma unroll
      for (int c = 0; c < 3; ++c) n2 = fmaf(acc[o4][c].x, acc[o4][c].x, fmaf(acc[o4][c].y, acc[o4][c].y, n2));
      gf = 1.f / (1.f + __expf(-(a.gate_a[o] * n2 + a.gate_b[o])));
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const size_t kk = (((size_t)o * 2 + par) * 3 + c) * Vh + i;
      if (OUT == OUT_GATE_TRAIN) a.pre[kk] = acc[o4][c];
      a.out[kk] = make_float2(acc[o4][c].x * gf, acc[o4][c].y * gf);
    }
  }
}

// The 8 -> 8 inference layer with its channel mixing on the tensor cores (BF16 operands, FP32
// accumulation). For each colour the mixing of one tap is a real GEMM of sites x 16 inputs (8 channels,
// re and im) by 16 x 16 (8 output channels, re and im; a complex weight w acts on (re, im) as the 2 x 2
// block [[w.x, w.y], [-w.y, w.x]]): per 16 sites, one m16n8k16 warp MMA per colour and 8-column half.
// The gathers are those of k_conv88: two lanes per site, each transporting four input channels; a step
// gathers four hops (both directions of two dimensions), so their loads are in flight together (the layer
// is bound by gather latency, not by its arithmetic). Each lane rounds its transported channels to BF16 and writes
// them, one 16-byte half row per colour, into its warp's shared-memory tile of 16 sites; ldmatrix then
// hands the MMA its A fragments (16 sites x 16 inputs per colour). The weights' B fragments are built
// once per block in shared memory. Sums and the gate are FP32.
__device__ __forceinline__ unsigned pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const unsigned*>(&v);
}

__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
  asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
               "{%0, %1, %2, %3};"
               : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
               : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void ldmatrix_x4(unsigned (&a)[4], const void* smem_row) {
  const unsigned addr = (unsigned)__cvta_generic_to_shared(smem_row);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
               : "=r"(a[0]), "=r"(a[1]), "=r"(a[2]), "=r"(a[3])
               : "r"(addr)
               : "memory");
}

// A tile row is one site's 16 BF16 inputs of one colour: two 16-byte halves (channels 0-3, 4-7). The
// half index is XOR-ed with bit 2 of the row, so the 8 rows an ldmatrix phase reads (32-byte stride)
// fall on distinct banks.
__device__ __forceinline__ int tc_half(int row, int half) { return half ^ ((row >> 2) & 1); }

template <int OUT>
__global__ void __launch_bounds__(kThreads, 3) k_conv88_tc(ConvArgs a) {
  if (a.st && !gate_open(a.st, a.gate)) return;
  constexpr int kWarps = kThreads / 32;
  // B fragments [tap][nt][half][lane]: rows k = 2 ci + comp (ci = t, t + 4 for half 0, 1), column n = g of
  // each 8-column half nt, i.e. output channel o = 4 nt + g / 2, component g % 2 (lane = 4 g + t)
  __shared__ unsigned sB[NT][2][2][32];
  __shared__ __align__(16) uint4 sA[kWarps][4][3][16][2];  // [warp][hop][colour][site][half], BF16 inputs
  for (int e = threadIdx.x; e < NT * 2 * 2 * 32; e += blockDim.x) {
    const int l = e & 31, half = (e >> 5) & 1, nt = (e >> 6) & 1, tap = e >> 7;
    const int o = 4 * nt + (l >> 3), oc = (l >> 2) & 1;
    const float2 w = a.W[(tap * CH + o) * CH + (l & 3) + 4 * half];
    // (re, im) input component -> output component oc: re: (w.x, -w.y); im: (w.y, w.x)
    sB[tap][nt][half][l] = oc == 0 ? pack_bf16(w.x, -w.y) : pack_bf16(w.y, w.x);
  }
  __syncthreads();
  const Geom& g = a.g;
  const int Vh = g.Vh;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long nsites = (long)a.npar * Vh;
  const long site0 = ((long)blockIdx.x * kWarps + warp) * 16;  // the warp's first site
  // two lanes per site, as k_conv88: lane 2 s + h gathers and transports input channels 4 h .. 4 h + 3 of
  // site s (a site past the end reads site 0; its rows are not stored)
  const int sl = lane >> 1, h = lane & 1;
  const long site = site0 + sl;
  const long sv = site < nsites ? site : 0;
  const int par = a.par0 + (int)(sv / Vh), idx = (int)(sv % Vh);
  const int q = 1 - par;
  const Site st = site_of(g, idx, par);
  uint4(*tile)[3][16][2] = sA[warp];
  const int my_half = tc_half(sl, h);
  // ldmatrix: lane l addresses row l % 8 (+ 8 for matrices 1, 3) of half l / 16
  const int mrow = (lane & 7) + 8 * ((lane >> 3) & 1);
  const int mhalf = tc_half(mrow, lane >> 4);
  float acc[3][2][4];
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[c][nt][e] = 0.f;
  auto mma_tap = [&](int tap, int slot) {
    const unsigned b00 = sB[tap][0][0][lane], b01 = sB[tap][0][1][lane];
    const unsigned b10 = sB[tap][1][0][lane], b11 = sB[tap][1][1][lane];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      unsigned af[4];
      ldmatrix_x4(af, &tile[slot][c][mrow][mhalf]);
      mma_bf16_16816(acc[c][0], af, b00, b01);
      mma_bf16_16816(acc[c][1], af, b10, b11);
    }
  };
  // self tap: this lane's four channels at its site
  {
    unsigned w[3][4];
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float2 v = __ldg(a.in + (((size_t)(4 * h + k) * 2 + par) * 3 + c) * Vh + idx);
        w[c][k] = pack_bf16(v.x, v.y);
      }
#pragma unroll
    for (int c = 0; c < 3; ++c) tile[0][c][sl][my_half] = make_uint4(w[c][0], w[c][1], w[c][2], w[c][3]);
    __syncwarp();
    mma_tap(0, 0);
  }
  // hops: two directions, forward and backward, per step (four hops)
#pragma unroll 1
  for (int mp = 0; mp < 2; ++mp) {
    unsigned w[4][3][4];
#pragma unroll
    for (int hop = 0; hop < 4; ++hop) {
      const int mu = 2 * mp + (hop >> 1), dir = hop & 1;
      const int j = nbr(g, st, mu, dir == 0 ? +1 : -1);
      float2 u[9];
      if (dir == 0) load_link9(a.fat[par] + (size_t)mu * 9 * Vh, Vh, idx, u);  // F_mu(n)
      else load_link9(a.fat[q] + (size_t)mu * 9 * Vh, Vh, j, u);               // F_mu(n - mu)
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        float2 v[3], t[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) v[c] = __ldg(a.in + (((size_t)(4 * h + k) * 2 + q) * 3 + c) * Vh + j);
        apply_link(u, dir == 1, v, t);
#pragma unroll
        for (int c = 0; c < 3; ++c) w[hop][c][k] = pack_bf16(t[c].x, t[c].y);
      }
    }
    __syncwarp();  // the previous step's ldmatrix reads of this warp's tiles are done
#pragma unroll
    for (int hop = 0; hop < 4; ++hop)
#pragma unroll
      for (int c = 0; c < 3; ++c)
        tile[hop][c][sl][my_half] = make_uint4(w[hop][c][0], w[hop][c][1], w[hop][c][2], w[hop][c][3]);
    __syncwarp();
#pragma unroll
    for (int hop = 0; hop < 4; ++hop) mma_tap(1 + 4 * mp + hop, hop);
  }
  // epilogue: accumulator element (row g or g + 8, column 2 t + {0, 1}) of half nt is output channel
  // o = 4 nt + t, (re, im), at site site0 + g (+ 8)
  const int gq = lane >> 2, tq = lane & 3;
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const long s2 = site0 + gq + 8 * r;
    if (s2 >= nsites) continue;
    const int par2 = a.par0 + (int)(s2 / Vh), idx2 = (int)(s2 % Vh);
#pragma unroll
    for (int nt = 0; nt < 2; ++nt) {
      const int o = 4 * nt + tq;
      float2 v[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) v[c] = make_float2(acc[c][nt][2 * r], acc[c][nt][2 * r + 1]);
      float gf = 1.f;
      if (OUT == OUT_GATE_INFER) {
        float n2 = 0.f;
#pragma unroll
        for (int c = 0; c < 3; ++c) n2 = fmaf(v[c].x, v[c].x, fmaf(v[c].y, v[c].y, n2));
        gf = 1.f / (1.f + __expf(-(a.gate_a[o] * n2 + a.gate_b[o])));
      }
#pragma unroll
      for (int c = 0; c < 3; ++c)
        a.out[(((size_t)o * 2 + par2) * 3 + c) * Vh + idx2] = make_float2(v[c].x * gf, v[c].y * gf);
    }
  }
}

// ---------------------------------------------------------------------------
// training kernels
// ---------------------------------------------------------------------------
// gradient through the gate: given pre-activation a and dL/dh, write dL/da and
// accumulate dL/dgate_a, dL/dgate_b per channel (block partials [blk][2*CH])
__global__ void __launch_bounds__(kRedThreads) k_gate_bwd(const float2* __restrict__ pre, const float2* __restrict__ gh,
                                                          float2* __restrict__ ga, const float* gate_a,
                                                          const float* gate_b, int Vh, double* partials) {
  const int n = 2 * Vh;
  const int gid = blockIdx.x * blockDim.x + threadIdx.x;
  __shared__ double red[2 * CH][kRedThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int o = 0; o < CH; ++o) {
    double da = 0.0, db = 0.0;
    if (gid < n) {
      const int par = gid / Vh, i = gid % Vh;
      float2 h[3], g[3];
      float n2 = 0.f, proj = 0.f;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const size_t k = (((size_t)o * 2 + par) * 3 + c) * Vh + i;
        h[c] = pre[k];
        g[c] = gh[k];
        n2 = fmaf(h[c].x, h[c].x, fmaf(h[c].y, h[c].y, n2));
        proj = fmaf(h[c].x, g[c].x, fmaf(h[c].y, g[c].y, proj));
      }
      const float sg = 1.f / (1.f + __expf(-(gate_a[o] * n2 + gate_b[o])));
      const float gp = sg * (1.f - sg);
      const float coef = 2.f * gate_a[o] * gp * proj;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const size_t k = (((size_t)o * 2 + par) * 3 + c) * Vh + i;
        ga[k] = make_float2(sg * g[c].x + coef * h[c].x, sg * g[c].y + coef * h[c].y);
      }
      da = (double)(gp * n2 * proj);
      db = (double)(gp * proj);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      da += __shfl_down_sync(0xffffffffu, da, off);
      db += __shfl_down_sync(0xffffffffu, db, off);
    }
    if (lane == 0) {
      red[o][wid] = da;
      red[CH + o][wid] = db;
    }
  }
  __syncthreads();
  if (threadIdx.x < 2 * CH) {
    double s = 0.0;
    for (int w = 0; w < kRedThreads / 32; ++w) s += red[threadIdx.x][w];
    partials[(size_t)blockIdx.x * 2 * CH + threadIdx.x] = s;
  }
}

// the 9 tap fields of an input field, for every site: T[tap][ci][par][3][Vh]
template <int CIN, int IN>
__global__ void __launch_bounds__(kThreads, 4) k_taps(ConvArgs a, float2* __restrict__ T) {
  const Geom& g = a.g;
  const int Vh = g.Vh;
  const int gid = blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= 2 * Vh) return;
  const int par = gid / Vh, i = gid % Vh, q = 1 - par;
  const Site s = site_of(g, i, par);
  const float sc = (IN == IN_EVEN_SCALED) ? (float)*a.scale : 1.f;
  auto load_in = [&](int ci, int pp, int j, float2 (&v)[3]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      if (IN == IN_FULL) {
        v[c] = __ldg(a.in + (((size_t)ci * 2 + pp) * 3 + c) * Vh + j);
      } else {
        const float2 t = (pp == 0) ? __ldg(a.in + (size_t)c * Vh + j) : make_float2(0.f, 0.f);
        v[c] = make_float2(t.x * sc, t.y * sc);
      }
    }
  };
  auto store = [&](int tap, int ci, const float2 (&t)[3]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) T[((((size_t)tap * CIN + ci) * 2 + par) * 3 + c) * Vh + i] = t[c];
  };
#pragma unroll
  for (int ci = 0; ci < CIN; ++ci) {
    float2 v[3];
    load_in(ci, par, i, v);
    store(0, ci, v);
  }
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
#pragma unroll
    for (int dir = 0; dir < 2; ++dir) {
      const int j = nbr(g, s, mu, dir == 0 ? +1 : -1);
      float2 u[9];
      if (dir == 0) load_link9(a.fat[par] + (size_t)mu * 9 * Vh, Vh, i, u);
      else load_link9(a.fat[q] + (size_t)mu * 9 * Vh, Vh, j, u);
#pragma unroll
      for (int ci = 0; ci < CIN; ++ci) {
        float2 v[3], t[3];
        load_in(ci, q, j, v);
        apply_link(u, dir == 1, v, t);
        store(1 + 2 * mu + dir, ci, t);
      }
    }
  }
}

// weight gradient partials: dW[tap][o][ci] = sum_sites sum_c conj(T[tap][ci]) g[o]
// (block partials [blk][NT*COUT*CIN] complex, as two doubles each)
template <int CIN, int COUT>
__global__ void __launch_bounds__(kRedThreads) k_wgrad(const float2* __restrict__ T, const float2* __restrict__ G,
                                                       int Vh, int even_only, double* partials) {
  constexpr int NE = NT * COUT * CIN;
  constexpr int CHUNK = 16;
  __shared__ float2 sT[NT * CIN][3][CHUNK];
  __shared__ float2 sG[COUT][3][CHUNK];
  const int nsites = even_only ? Vh : 2 * Vh;
  double accr[(NE + kRedThreads - 1) / kRedThreads], acci[(NE + kRedThreads - 1) / kRedThreads];
#pragma unroll
  for (int k = 0; k < (NE + kRedThreads - 1) / kRedThreads; ++k) accr[k] = acci[k] = 0.0;
  for (int base = blockIdx.x * CHUNK; base < nsites; base += gridDim.x * CHUNK) {
    __syncthreads();
    for (int j = threadIdx.x; j < NT * CIN * 3 * CHUNK; j += blockDim.x) {
      const int sidx = j % CHUNK, c = (j / CHUNK) % 3, tc = j / (3 * CHUNK);
      const int site = base + sidx;
      float2 v = make_float2(0.f, 0.f);
      if (site < nsites) {
        const int par = site / Vh, i = site % Vh;
        v = T[(((size_t)tc * 2 + par) * 3 + c) * Vh + i];
      }
      sT[tc][c][sidx] = v;
    }
    for (int j = threadIdx.x; j < COUT * 3 * CHUNK; j += blockDim.x) {
      const int sidx = j % CHUNK, c = (j / CHUNK) % 3, o = j / (3 * CHUNK);
      const int site = base + sidx;
      float2 v = make_float2(0.f, 0.f);
      if (site < nsites) {
        const int par = site / Vh, i = site % Vh;
        v = G[(((size_t)o * 2 + par) * 3 + c) * Vh + i];
      }
      sG[o][c][sidx] = v;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < (NE + kRedThreads - 1) / kRedThreads; ++k) {
      const int e = threadIdx.x + k * kRedThreads;
      if (e >= NE) continue;
      const int ci = e % CIN, o = (e / CIN) % COUT, tap = e / (CIN * COUT);
      float sr = 0.f, si = 0.f;
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int j = 0; j < CHUNK; ++j) {
          const float2 t = sT[tap * CIN + ci][c][j], gg = sG[o][c][j];
          sr = fmaf(t.x, gg.x, fmaf(t.y, gg.y, sr));   // Re(conj(t) g)
          si = fmaf(t.x, gg.y, fmaf(-t.y, gg.x, si));  // Im(conj(t) g)
        }
      accr[k] += sr;
      acci[k] += si;
    }
  }
#pragma unroll
  for (int k = 0; k < (NE + kRedThreads - 1) / kRedThreads; ++k) {
    const int e = threadIdx.x + k * kRedThreads;
    if (e < NE) {
      partials[((size_t)blockIdx.x * NE + e) * 2] = accr[k];
      partials[((size_t)blockIdx.x * NE + e) * 2 + 1] = acci[k];
    }
  }
}

// grad[off + j] += sum over blocks of partials[blk][j] (index order)
__global__ void k_sum_partials(const double* __restrict__ partials, int nblk, int n, float* grad, int off) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += partials[(size_t)b * n + j];
  grad[off + j] += (float)s;
}

// generic FP32 two-vector dot products over even vectors [3][Vh]: sum Re<a, b>
__global__ void __launch_bounds__(kRedThreads) k_dot2(const float2* a1, const float2* b1, const float2* a2,
                                                      const float2* b2, int Vh, double* partials) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double u = 0.0, v = 0.0;
  if (i < Vh) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const size_t k = (size_t)c * Vh + i;
      const float2 x = a1[k], y = b1[k];
      u += (double)x.x * y.x + (double)x.y * y.y;
      if (a2) {
        const float2 p = a2[k], qv = b2[k];
        v += (double)p.x * qv.x + (double)p.y * qv.y;
      }
    }
  }
  block_partial2(u, v, partials);
}

// d = z - e
__global__ void k_sub(const float2* z, const float2* e, float2* d, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) d[i] = make_float2(z[i].x - e[i].x, z[i].y - e[i].y);
}

// g3 (even, full-lattice layout [1][2][3][Vh], odd = 0) = coef * Ad with coef = 2 / (<e,r> s)
__global__ void k_dz(const float2* Ad, float2* g3, int Vh, const double* scal) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= 3 * Vh) return;
  const float coef = (float)(2.0 / (scal[2] * scal[0]));
  const int c = j / Vh, i = j % Vh;
  g3[((size_t)0 * 3 + c) * Vh + i] = make_float2(coef * Ad[j].x, coef * Ad[j].y);
  g3[((size_t)1 * 3 + c) * Vh + i] = make_float2(0.f, 0.f);
}

// two-sum finisher into nn scalars: mode 0: scal[0] = s = sqrt(3Vh/a), scal[1] = 1/s (input scale);
// mode 1: scal[2] = <e,r> = b, scal[3] += <d,Ad>/<e,r> = a/b (loss)
__global__ void k_nn_finish(const double* partials, int n, double* scal, int mode, int Vh) {
  double a = 0.0, b = 0.0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    a += partials[j];
    b += partials[n + j];
  }
  a = block_sum(a);
  b = block_sum(b);
  if (threadIdx.x == 0) {
    if (mode == 0) {
      scal[0] = (a > 0) ? sqrt(3.0 * Vh / a) : 0.0;
      scal[1] = (a > 0) ? 1.0 / scal[0] : 0.0;
    } else {
      scal[2] = b;
      scal[3] += a / b;
    }
  }
}

// Adam step over all parameters; grad holds the sum over the batch (divided by nb)
__global__ void k_adam(float* w, const float* grad, float* m, float* v, int n, float lr, float b1, float b2, float eps,
                       int t, float inv_nb) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const float g = grad[j] * inv_nb;
  const float mj = b1 * m[j] + (1.f - b1) * g;
  const float vj = b2 * v[j] + (1.f - b2) * g * g;
  m[j] = mj;
  v[j] = vj;
  const float mh = mj / (1.f - powf(b1, (float)t));
  const float vh = vj / (1.f - powf(b2, (float)t));
  w[j] -= lr * mh / (sqrtf(vh) + eps);
}

// forward weights (BF16-rounded, FP32 copy) and adjoint weights from the FP32 master:
// fwd[l] = bf16(W_l); adj[l][tap'][ci][o] = conj(fwd[l][tap][o][ci]) with tap' = self, fwd <-> bwd swapped
__global__ void k_round_weights(const float* master, float2* fwd, float2* adj) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= NWEIGHT) return;
  const float re = __bfloat162float(__float2bfloat16_rn(master[2 * j]));
  const float im = __bfloat162float(__float2bfloat16_rn(master[2 * j + 1]));
  fwd[j] = make_float2(re, im);
  // locate layer, tap, o, ci
  int base, cin, cout, k;
  if (j < OFF_W2 / 2) { base = 0; cin = 1; cout = CH; k = j; }
  else if (j < OFF_W3 / 2) { base = OFF_W2 / 2; cin = CH; cout = CH; k = j - base; }
  else { base = OFF_W3 / 2; cin = CH; cout = 1; k = j - base; }
  const int ci = k % cin, o = (k / cin) % cout, tap = k / (cin * cout);
  const int tap2 = (tap == 0) ? 0 : ((tap & 1) ? tap + 1 : tap - 1);
  // adjoint layer maps cout channels -> cin channels: [tap2][ci][o]
  adj[base + (tap2 * cin + ci) * cout + o] = make_float2(re, -im);
}

int nn_grid(int n) { return (n + kThreads - 1) / kThreads; }

}  // namespace

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct sqcg_nn {
  sqcg_ctx* ctx;
  float* master;   // [NPARAM] FP32
  float2* wfwd;    // [NWEIGHT] BF16-rounded forward weights in FP32
  float2* wadj;    // [NWEIGHT] adjoint-layer weights
  float* grad;     // [NPARAM]
  float* adam_m;
  float* adam_v;
  int adam_t;
  double* scal;    // [8]: s, 1/s, <e,r>, loss sum
  double* partials;
  size_t npartials;
  float2 *h1, *h2;         // inference / training activations [CH][2][3][Vh]
  float2 *a1, *a2;         // training pre-activations
  float2 *g1, *g2, *g3;    // training gradients ([CH][2][3][Vh], g3 [1][2][3][Vh])
  float2* T;               // training taps [9][CH][2][3][Vh]
  float2 *d, *Ad, *tmp, *zbuf;  // even FP32 vectors (training) / odd temp
  float2 *r_old, *z;       // flexible CG vectors
  // the captured flexible-CG loop, reused while b, x and the links stay the same
  cudaGraphExec_t fcg_exec;
  cudaGraphConditionalHandle fcg_hw, fcg_hif;
  const void* fcg_b;
  void* fcg_x;
  unsigned long long fcg_gen;
  bool train_ready;
  int loss_norm;           // 1: A-norm of the error, 2: A^2-norm (preconditioned residual)
  int mixing;              // inference 8 -> 8 layer: SQCG_NN_MIX_FP32 (CUDA cores) or SQCG_NN_MIX_BF16 (tensor cores)
};

namespace {

int conv_launch(sqcg_nn* nn, int layer, bool adjoint, int in_mode, int out_mode, const float2* in, float2* out,
                float2* pre, int par0, int npar, const SolverState* st, int gate, const double* scale,
                cudaStream_t s) {
  sqcg_ctx* ctx = nn->ctx;
  ConvArgs a;
  a.g = ctx->g;
  const size_t Vh = ctx->g.Vh;
  a.fat[0] = ctx->fat32;
  a.fat[1] = ctx->fat32 + 4 * 9 * Vh;
  a.in = in;
  a.out = out;
  a.pre = pre;
  const float2* W = adjoint ? nn->wadj : nn->wfwd;
  const int offs[3] = {OFF_W1 / 2, OFF_W2 / 2, OFF_W3 / 2};
  a.W = W + offs[layer];
  a.gate_a = nn->master + OFF_G + (layer == 0 ? 0 : 2 * CH);
  a.gate_b = a.gate_a + CH;
  a.scale = scale;
  a.st = st;
  a.gate = gate;
  a.par0 = par0;
  a.npar = npar;
  const int grid = nn_grid(npar * (int)Vh);
  const int grid2 = nn_grid(2 * npar * (int)Vh);  // the two-lane 8 -> 8 kernel
  // channel counts of the (possibly adjoint) layer
  int cin = (layer == 0) ? 1 : CH, cout = (layer == 2) ? 1 : CH;
  if (adjoint) { const int t = cin; cin = cout; cout = t; }
  if (cin == 1 && cout == CH && in_mode == IN_EVEN_SCALED && out_mode == OUT_GATE_INFER)
    k_conv<1, CH, IN_EVEN_SCALED, OUT_GATE_INFER><<<grid, kThreads, 0, s>>>(a);
  else if (cin == 1 && cout == CH && in_mode == IN_EVEN_SCALED && out_mode == OUT_GATE_TRAIN)
    k_conv<1, CH, IN_EVEN_SCALED, OUT_GATE_TRAIN><<<grid, kThreads, 0, s>>>(a);
  else if (cin == CH && cout == CH && in_mode == IN_FULL && out_mode == OUT_GATE_INFER && !adjoint &&
           nn->mixing == SQCG_NN_MIX_BF16)
    k_conv88_tc<OUT_GATE_INFER><<<grid_for(npar * (int)Vh, kThreads / 2), kThreads, 0, s>>>(a);
  else if (cin == CH && cout == CH && in_mode == IN_FULL && out_mode == OUT_GATE_INFER)
    k_conv88<OUT_GATE_INFER><<<grid2, kThreads, 0, s>>>(a);
  else if (cin == CH && cout == CH && in_mode == IN_FULL && out_mode == OUT_GATE_TRAIN)
    k_conv88<OUT_GATE_TRAIN><<<grid2, kThreads, 0, s>>>(a);
  else if (cin == CH && cout == CH && in_mode == IN_FULL && out_mode == OUT_FULL)
    k_conv88<OUT_FULL><<<grid2, kThreads, 0, s>>>(a);
  else if (cin == CH && cout == 1 && in_mode == IN_FULL && out_mode == OUT_EVEN_SCALED)
    k_conv<CH, 1, IN_FULL, OUT_EVEN_SCALED><<<grid, kThreads, 0, s>>>(a);
  else if (cin == 1 && cout == CH && in_mode == IN_FULL && out_mode == OUT_FULL)
    k_conv<1, CH, IN_FULL, OUT_FULL><<<grid, kThreads, 0, s>>>(a);
  else
    return SQCG_ERR_INVALID_ARG;
  SQCG_CUDA_TRY(cudaGetLastError());
  return SQCG_OK;
}

// z = N(r) on the even sites (inference). scale[0] must hold s, scale[1] 1/s.
int nn_forward_infer(sqcg_nn* nn, const float2* r, float2* z, const double* scale, const SolverState* st, int gate,
                     cudaStream_t s) {
  SQCG_TRY(conv_launch(nn, 0, false, IN_EVEN_SCALED, OUT_GATE_INFER, r, nn->h1, nullptr, 0, 2, st, gate, scale, s));
  SQCG_TRY(conv_launch(nn, 1, false, IN_FULL, OUT_GATE_INFER, nn->h1, nn->h2, nullptr, 0, 2, st, gate, nullptr, s));
  SQCG_TRY(conv_launch(nn, 2, false, IN_FULL, OUT_EVEN_SCALED, nn->h2, z, nullptr, 0, 1, st, gate, scale + 1, s));
  return SQCG_OK;
}

// scale of r into scal[0..1] (no solver state involved)
int nn_input_scale(sqcg_nn* nn, const float2* r, cudaStream_t s) {
  const int Vh = nn->ctx->g.Vh, grid = (Vh + kRedThreads - 1) / kRedThreads;
  k_dot2<<<grid, kRedThreads, 0, s>>>(r, r, nullptr, nullptr, Vh, nn->partials);
  k_nn_finish<<<1, kRedThreads, 0, s>>>(nn->partials, grid, nn->scal, 0, Vh);
  SQCG_CUDA_TRY(cudaGetLastError());
  return SQCG_OK;
}

int nn_refresh_weights(sqcg_nn* nn, cudaStream_t s) {
  k_round_weights<<<(NWEIGHT + 255) / 256, 256, 0, s>>>(nn->master, nn->wfwd, nn->wadj);
  SQCG_CUDA_TRY(cudaGetLastError());
  return SQCG_OK;
}

int nn_alloc_train(sqcg_nn* nn) {
  if (nn->train_ready) return SQCG_OK;
  const size_t Vh = nn->ctx->g.Vh;
  const size_t full = (size_t)CH * 2 * 3 * Vh;
  bool ok = cudaMalloc((void**)&nn->a1, full * sizeof(float2)) == cudaSuccess &&
            cudaMalloc((void**)&nn->a2, full * sizeof(float2)) == cudaSuccess &&
            cudaMalloc((void**)&nn->g1, full * sizeof(float2)) == cudaSuccess &&
            cudaMalloc((void**)&nn->g2, full * sizeof(float2)) == cudaSuccess &&
            cudaMalloc((void**)&nn->g3, 2 * 3 * Vh * sizeof(float2)) == cudaSuccess &&
            cudaMalloc((void**)&nn->T, (size_t)NT * full * sizeof(float2)) == cudaSuccess &&
            cudaMalloc((void**)&nn->d, 3 * Vh * sizeof(float2)) == cudaSuccess &&
            cudaMalloc((void**)&nn->Ad, 3 * Vh * sizeof(float2)) == cudaSuccess &&
            cudaMalloc((void**)&nn->tmp, 3 * Vh * sizeof(float2)) == cudaSuccess &&
            cudaMalloc((void**)&nn->zbuf, 3 * Vh * sizeof(float2)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    return SQCG_ERR_NO_MEMORY;
  }
  nn->train_ready = true;
  return SQCG_OK;
}

// weight-gradient contribution of one layer: grad[off..] += sum_sites conj(taps(h)) g
template <int CIN, int COUT>
int wgrad(sqcg_nn* nn, int in_mode, const float2* h, const float2* g, int even_only, int off, cudaStream_t s) {
  sqcg_ctx* ctx = nn->ctx;
  const int Vh = ctx->g.Vh;
  ConvArgs a = {};
  a.g = ctx->g;
  a.fat[0] = ctx->fat32;
  a.fat[1] = ctx->fat32 + 4 * 9 * (size_t)Vh;
  a.in = h;
  a.scale = nn->scal;
  if (in_mode == IN_FULL) k_taps<CIN, IN_FULL><<<nn_grid(2 * Vh), kThreads, 0, s>>>(a, nn->T);
  else k_taps<CIN, IN_EVEN_SCALED><<<nn_grid(2 * Vh), kThreads, 0, s>>>(a, nn->T);
  SQCG_CUDA_TRY(cudaGetLastError());
  constexpr int NE = NT * COUT * CIN;
  const int nsites = even_only ? Vh : 2 * Vh;
  int nblk = (nsites + 15) / 16;
  const int maxblk = (int)(nn->npartials / (2 * NE));
  if (nblk > maxblk) nblk = maxblk;
  if (nblk > 1024) nblk = 1024;
  k_wgrad<CIN, COUT><<<nblk, kRedThreads, 0, s>>>(nn->T, g, Vh, even_only, nn->partials);
  k_sum_partials<<<(2 * NE + 255) / 256, 256, 0, s>>>(nn->partials, nblk, 2 * NE, nn->grad, off);
  SQCG_CUDA_TRY(cudaGetLastError());
  return SQCG_OK;
}

int gate_bwd(sqcg_nn* nn, int layer, const float2* pre, const float2* gh, float2* ga, cudaStream_t s) {
  const int Vh = nn->ctx->g.Vh, grid = (2 * Vh + kRedThreads - 1) / kRedThreads;
  const float* gp = nn->master + OFF_G + (layer == 0 ? 0 : 2 * CH);
  k_gate_bwd<<<grid, kRedThreads, 0, s>>>(pre, gh, ga, gp, gp + CH, Vh, nn->partials);
  k_sum_partials<<<1, 64, 0, s>>>(nn->partials, grid, 2 * CH, nn->grad, OFF_G + (layer == 0 ? 0 : 2 * CH));
  SQCG_CUDA_TRY(cudaGetLastError());
  return SQCG_OK;
}

// forward (keeping activations), loss and gradient for one pair; grad += dL/dparams, scal[3] += loss
int nn_pair(sqcg_nn* nn, double sigma, const float2* r, const float2* e, cudaStream_t s) {
  sqcg_ctx* ctx = nn->ctx;
  const int Vh = ctx->g.Vh;
  SQCG_TRY(nn_input_scale(nn, r, s));
  SQCG_TRY(conv_launch(nn, 0, false, IN_EVEN_SCALED, OUT_GATE_TRAIN, r, nn->h1, nn->a1, 0, 2, nullptr, 0, nn->scal, s));
  SQCG_TRY(conv_launch(nn, 1, false, IN_FULL, OUT_GATE_TRAIN, nn->h1, nn->h2, nn->a2, 0, 2, nullptr, 0, nullptr, s));
  SQCG_TRY(conv_launch(nn, 2, false, IN_FULL, OUT_EVEN_SCALED, nn->h2, nn->zbuf, nullptr, 0, 1, nullptr, 0,
                       nn->scal + 1, s));
  // d = z - e; Ad = (sigma - D_eo D_oe) d in FP32; <d,Ad>, <e,r>
  k_sub<<<nn_grid(3 * Vh), kThreads, 0, s>>>(nn->zbuf, e, nn->d, 3 * Vh);
  DslashLaunch L = {};
  L.out_parity = 1; L.prec = L.out_prec = SQCG_F32; L.epi = EPI_PLAIN; L.in = nn->d; L.out = nn->tmp;
  SQCG_TRY(launch_dslash(ctx, L, s));
  L.out_parity = 0; L.epi = EPI_NORMAL; L.in = nn->tmp; L.out = nn->Ad; L.y = nn->d; L.sigma = sigma;
  SQCG_TRY(launch_dslash(ctx, L, s));
  const int grid = (Vh + kRedThreads - 1) / kRedThreads;
  if (nn->loss_norm == 2) {
    // L = <Ad, Ad> / <r, r>; dL/dz = 2 A (A d) / <r, r>   (A e = r: the preconditioned residual)
    L = DslashLaunch{};
    L.out_parity = 1; L.prec = L.out_prec = SQCG_F32; L.epi = EPI_PLAIN; L.in = nn->Ad; L.out = nn->tmp;
    SQCG_TRY(launch_dslash(ctx, L, s));
    L.out_parity = 0; L.epi = EPI_NORMAL; L.in = nn->tmp; L.out = nn->zbuf; L.y = nn->Ad; L.sigma = sigma;
    SQCG_TRY(launch_dslash(ctx, L, s));
    k_dot2<<<grid, kRedThreads, 0, s>>>(nn->Ad, nn->Ad, r, r, Vh, nn->partials);
    k_nn_finish<<<1, kRedThreads, 0, s>>>(nn->partials, grid, nn->scal, 1, Vh);
    k_dz<<<nn_grid(3 * Vh), kThreads, 0, s>>>(nn->zbuf, nn->g3, Vh, nn->scal);
  } else {
    // L = <d, A d> / <e, r>; dL/dz = 2 A d / <e, r>
    k_dot2<<<grid, kRedThreads, 0, s>>>(nn->d, nn->Ad, e, r, Vh, nn->partials);
    k_nn_finish<<<1, kRedThreads, 0, s>>>(nn->partials, grid, nn->scal, 1, Vh);
    k_dz<<<nn_grid(3 * Vh), kThreads, 0, s>>>(nn->Ad, nn->g3, Vh, nn->scal);
  }
  SQCG_CUDA_TRY(cudaGetLastError());
  // layer 3: dW3, dL/dh2
  SQCG_TRY((wgrad<CH, 1>(nn, IN_FULL, nn->h2, nn->g3, 1, OFF_W3, s)));
  SQCG_TRY(conv_launch(nn, 2, true, IN_FULL, OUT_FULL, nn->g3, nn->g2, nullptr, 0, 2, nullptr, 0, nullptr, s));
  // gate 2, layer 2
  SQCG_TRY(gate_bwd(nn, 1, nn->a2, nn->g2, nn->g2, s));
  SQCG_TRY((wgrad<CH, CH>(nn, IN_FULL, nn->h1, nn->g2, 0, OFF_W2, s)));
  SQCG_TRY(conv_launch(nn, 1, true, IN_FULL, OUT_FULL, nn->g2, nn->g1, nullptr, 0, 2, nullptr, 0, nullptr, s));
  // gate 1, layer 1
  SQCG_TRY(gate_bwd(nn, 0, nn->a1, nn->g1, nn->g1, s));
  SQCG_TRY((wgrad<1, CH>(nn, IN_EVEN_SCALED, r, nn->g1, 0, OFF_W1, s)));
  return SQCG_OK;
}

}  // namespace

extern "C" {

int sqcg_nn_create(sqcg_ctx* ctx, sqcg_nn** out) {
  if (!ctx || !out) return SQCG_ERR_INVALID_ARG;
  *out = nullptr;
  if (!ctx->have_links) return SQCG_ERR_NO_LINKS;
  sqcg_nn* nn = (sqcg_nn*)calloc(1, sizeof(sqcg_nn));
  if (!nn) return SQCG_ERR_NO_MEMORY;
  nn->ctx = ctx;
  nn->loss_norm = 1;
  const size_t Vh = ctx->g.Vh;
  const size_t full = (size_t)CH * 2 * 3 * Vh;
  // partials: enough for the largest reduction (weight gradients: 1024 blocks x 1152 doubles)
  nn->npartials = (size_t)1024 * 2 * NT * CH * CH;
  const size_t red2 = 2 * ((2 * Vh + kRedThreads - 1) / kRedThreads) * 2 * CH;
  if (red2 > nn->npartials) nn->npartials = red2;
  bool ok = cudaMalloc((void**)&nn->master, NPARAM * sizeof(float)) == cudaSuccess &&
            cudaMalloc((void**)&nn->wfwd, NWEIGHT * sizeof(float2)) == cudaSuccess &&
            cudaMalloc((void**)&nn->wadj, NWEIGHT * sizeof(float2)) == cudaSuccess &&
            cudaMalloc((void**)&nn->grad, NPARAM * sizeof(float)) == cudaSuccess &&
            cudaMalloc((void**)&nn->adam_m, NPARAM * sizeof(float)) == cudaSuccess &&
            cudaMalloc((void**)&nn->adam_v, NPARAM * sizeof(float)) == cudaSuccess &&
            cudaMalloc((void**)&nn->scal, 8 * sizeof(double)) == cudaSuccess &&
            cudaMalloc((void**)&nn->partials, nn->npartials * sizeof(double)) == cudaSuccess &&
            cudaMalloc((void**)&nn->h1, full * sizeof(float2)) == cudaSuccess &&
            cudaMalloc((void**)&nn->h2, full * sizeof(float2)) == cudaSuccess &&
            cudaMalloc((void**)&nn->r_old, 3 * Vh * sizeof(float2)) == cudaSuccess &&
            cudaMalloc((void**)&nn->z, 3 * Vh * sizeof(float2)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    sqcg_nn_destroy(nn);
    return SQCG_ERR_NO_MEMORY;
  }
  cudaStream_t s = ctx->stream;
  SQCG_CUDA_TRY(cudaMemsetAsync(nn->master, 0, NPARAM * sizeof(float), s));
  SQCG_CUDA_TRY(cudaMemsetAsync(nn->adam_m, 0, NPARAM * sizeof(float), s));
  SQCG_CUDA_TRY(cudaMemsetAsync(nn->adam_v, 0, NPARAM * sizeof(float), s));
  SQCG_CUDA_TRY(cudaMemsetAsync(nn->scal, 0, 8 * sizeof(double), s));
  SQCG_TRY(nn_refresh_weights(nn, s));
  *out = nn;
  return SQCG_OK;
}

int sqcg_nn_destroy(sqcg_nn* nn) {
  if (!nn) return SQCG_OK;
  // the context may already be gone: wait for the device, not for the context's stream
  cudaDeviceSynchronize();
  if (nn->fcg_exec) cudaGraphExecDestroy(nn->fcg_exec);
  void* bufs[] = {nn->master, nn->wfwd, nn->wadj, nn->grad, nn->adam_m, nn->adam_v, nn->scal, nn->partials,
                  nn->h1, nn->h2, nn->a1, nn->a2, nn->g1, nn->g2, nn->g3, nn->T, nn->d, nn->Ad, nn->tmp,
                  nn->zbuf, nn->r_old, nn->z};
  for (void* b : bufs) cudaFree(b);
  free(nn);
  return SQCG_OK;
}

int sqcg_nn_nparams(void) { return NPARAM; }

int sqcg_nn_set_loss(sqcg_nn* nn, int norm) {
  if (!nn || (norm != 1 && norm != 2)) return SQCG_ERR_INVALID_ARG;
  nn->loss_norm = norm;
  return SQCG_OK;
}

int sqcg_nn_set_mixing(sqcg_nn* nn, int mode) {
  if (!nn || (mode != SQCG_NN_MIX_FP32 && mode != SQCG_NN_MIX_BF16)) return SQCG_ERR_INVALID_ARG;
  if (mode != nn->mixing && nn->fcg_exec) {  // the captured loop holds the other kernel
    cudaStreamSynchronize(nn->ctx->stream);
    cudaGraphExecDestroy(nn->fcg_exec);
    nn->fcg_exec = nullptr;
  }
  nn->mixing = mode;
  return SQCG_OK;
}

int sqcg_nn_set_params(sqcg_nn* nn, const float* params) {
  if (!nn || !params) return SQCG_ERR_INVALID_ARG;
  for (int j = 0; j < NPARAM; ++j)
    if (!isfinite(params[j])) return SQCG_ERR_INVALID_ARG;
  cudaStream_t s = nn->ctx->stream;
  SQCG_CUDA_TRY(cudaMemcpyAsync(nn->master, params, NPARAM * sizeof(float), cudaMemcpyHostToDevice, s));
  SQCG_CUDA_TRY(cudaMemsetAsync(nn->adam_m, 0, NPARAM * sizeof(float), s));
  SQCG_CUDA_TRY(cudaMemsetAsync(nn->adam_v, 0, NPARAM * sizeof(float), s));
  nn->adam_t = 0;
  SQCG_TRY(nn_refresh_weights(nn, s));
  SQCG_CUDA_TRY(cudaStreamSynchronize(s));
  return SQCG_OK;
}

int sqcg_nn_get_params(const sqcg_nn* nn, float* params, int bf16_rounded) {
  if (!nn || !params) return SQCG_ERR_INVALID_ARG;
  cudaStream_t s = nn->ctx->stream;
  SQCG_CUDA_TRY(cudaMemcpyAsync(params, nn->master, NPARAM * sizeof(float), cudaMemcpyDeviceToHost, s));
  if (bf16_rounded)
    SQCG_CUDA_TRY(cudaMemcpyAsync(params, nn->wfwd, NWEIGHT * sizeof(float2), cudaMemcpyDeviceToHost, s));
  SQCG_CUDA_TRY(cudaStreamSynchronize(s));
  return SQCG_OK;
}

int sqcg_nn_apply(sqcg_nn* nn, const void* r, void* z) {
  if (!nn || !r || !z || r == z) return SQCG_ERR_INVALID_ARG;
  cudaStream_t s = nn->ctx->stream;
  SQCG_TRY(nn_input_scale(nn, (const float2*)r, s));
  return nn_forward_infer(nn, (const float2*)r, (float2*)z, nn->scal, nullptr, GATE_NONE, s);
}

int sqcg_nn_loss_grad(sqcg_nn* nn, double sigma, const void* r, const void* e, double* loss, float* grad) {
  if (!nn || !r || !e || !(sigma >= 0)) return SQCG_ERR_INVALID_ARG;
  SQCG_TRY(nn_alloc_train(nn));
  cudaStream_t s = nn->ctx->stream;
  SQCG_CUDA_TRY(cudaMemsetAsync(nn->grad, 0, NPARAM * sizeof(float), s));
  SQCG_CUDA_TRY(cudaMemsetAsync(nn->scal + 3, 0, sizeof(double), s));
  SQCG_TRY(nn_pair(nn, sigma, (const float2*)r, (const float2*)e, s));
  double sc[4];
  SQCG_CUDA_TRY(cudaMemcpyAsync(sc, nn->scal, sizeof(sc), cudaMemcpyDeviceToHost, s));
  if (grad) SQCG_CUDA_TRY(cudaMemcpyAsync(grad, nn->grad, NPARAM * sizeof(float), cudaMemcpyDeviceToHost, s));
  SQCG_CUDA_TRY(cudaStreamSynchronize(s));
  if (loss) *loss = sc[3];
  return SQCG_OK;
}

int sqcg_nn_train(sqcg_nn* nn, double sigma, int npairs, const void* r, const void* e, int steps, int batch,
                  double lr, unsigned long long seed, double* loss_first, double* loss_last) {
  if (!nn || !r || !e || npairs < 1 || steps < 1 || batch < 1 || !(lr > 0) || !(sigma >= 0))
    return SQCG_ERR_INVALID_ARG;
  SQCG_TRY(nn_alloc_train(nn));
  cudaStream_t s = nn->ctx->stream;
  const size_t vec = (size_t)3 * nn->ctx->g.Vh;
  unsigned long long state = seed ? seed : 0x9e3779b97f4a7c15ULL;
  double first = 0.0, last = 0.0;
  for (int step = 0; step < steps; ++step) {
    SQCG_CUDA_TRY(cudaMemsetAsync(nn->grad, 0, NPARAM * sizeof(float), s));
    SQCG_CUDA_TRY(cudaMemsetAsync(nn->scal + 3, 0, sizeof(double), s));
    for (int b = 0; b < batch; ++b) {
      state = state * 6364136223846793005ULL + 1442695040888963407ULL;  // LCG (Knuth MMIX constants)
      const int k = (int)((state >> 33) % (unsigned long long)npairs);
      SQCG_TRY(nn_pair(nn, sigma, (const float2*)r + k * vec, (const float2*)e + k * vec, s));
    }
    nn->adam_t += 1;
    k_adam<<<(NPARAM + 255) / 256, 256, 0, s>>>(nn->master, nn->grad, nn->adam_m, nn->adam_v, NPARAM, (float)lr,
                                                0.9f, 0.999f, 1e-8f, nn->adam_t, 1.f / batch);
    SQCG_CUDA_TRY(cudaGetLastError());
    SQCG_TRY(nn_refresh_weights(nn, s));
    if (step == 0 || step == steps - 1) {
      double l;
      SQCG_CUDA_TRY(cudaMemcpyAsync(&l, nn->scal + 3, sizeof(double), cudaMemcpyDeviceToHost, s));
      SQCG_CUDA_TRY(cudaStreamSynchronize(s));
      if (step == 0) first = l / batch;
      last = l / batch;
    }
  }
  if (loss_first) *loss_first = first;
  if (loss_last) *loss_last = last;
  return SQCG_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// flexible CG
// ---------------------------------------------------------------------------
namespace {

// r_old = r; x += alpha p (x FP64); r -= alpha q; |r|^2 partials. Held to 5 blocks a SM, the residency that
// sizes the one-wave grid of blas_grid() (56 registers unbounded fit 4: 1.25 waves).
__global__ void __launch_bounds__(kRedThreads, 5) k_fcg_update(double2* __restrict__ x, float2* __restrict__ r,
                                                            float2* __restrict__ r_old, const float2* __restrict__ p,
                                                            const float2* __restrict__ q, int Vh, SolverState* st,
                                                            double* partials) {
  if (!gate_open(st, GATE_ITER)) return;
  const double alpha = st->alpha;
  const float fa = (float)alpha;
  double nrm = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < Vh; i += gridDim.x * blockDim.x) {
    // every colour component is loaded before any store, so the loads overlap
    float2 pc[3], qc[3], rc[3];
    double2 xc[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const size_t k = (size_t)c * Vh + i;
      pc[c] = p[k];
      qc[c] = q[k];
      rc[c] = r[k];
      xc[c] = x[k];
    }
    float part = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const size_t k = (size_t)c * Vh + i;
      r_old[k] = rc[c];
      xc[c].x = fma(alpha, (double)pc[c].x, xc[c].x);
      xc[c].y = fma(alpha, (double)pc[c].y, xc[c].y);
      x[k] = xc[c];
      rc[c].x = fmaf(-fa, qc[c].x, rc[c].x);
      rc[c].y = fmaf(-fa, qc[c].y, rc[c].y);
      r[k] = rc[c];
      part = fmaf(rc[c].x, rc[c].x, fmaf(rc[c].y, rc[c].y, part));
    }
    nrm += (double)part;
  }
  block_partial(nrm, partials);
}

// <z, r> and <z, r_old> partials: each site's sum in FP32, the sums over sites in FP64
__global__ void __launch_bounds__(kRedThreads) k_fcg_dots(const float2* __restrict__ z, const float2* __restrict__ r,
                                                          const float2* __restrict__ r_old, int Vh,
                                                          const SolverState* st, double* partials) {
  if (!gate_open(st, GATE_ITER)) return;
  double a = 0.0, b = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < Vh; i += gridDim.x * blockDim.x) {
    float2 zc[3], rc[3], oc[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const size_t k = (size_t)c * Vh + i;
      zc[c] = z[k];
      rc[c] = r[k];
      oc[c] = r_old[k];
    }
    float pa = 0.f, pb = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      pa = fmaf(zc[c].x, rc[c].x, fmaf(zc[c].y, rc[c].y, pa));
      pb = fmaf(zc[c].x, oc[c].x, fmaf(zc[c].y, oc[c].y, pb));
    }
    a += (double)pa;
    b += (double)pb;
  }
  block_partial2(a, b, partials);
}

// |r|^2 partials for the network input scale (gated)
__global__ void __launch_bounds__(kRedThreads) k_norm_gated(const float2* __restrict__ r, int Vh, const SolverState* st,
                                                            double* partials) {
  if (!gate_open(st, GATE_ITER)) return;
  double a = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < Vh; i += gridDim.x * blockDim.x) {
    float2 v[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) v[c] = r[(size_t)c * Vh + i];
    float part = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) part = fmaf(v[c].x, v[c].x, fmaf(v[c].y, v[c].y, part));
    a += (double)part;
  }
  block_partial(a, partials);
}

// p = z + beta p over the 3 Vh colour components
__global__ void __launch_bounds__(kRedThreads) k_fcg_xpay(const float2* __restrict__ z, float2* __restrict__ p, int n,
                                                          const SolverState* st) {
  if (!gate_open(st, GATE_ITER)) return;
  const float b = (float)st->beta;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float2 zc = z[i];
    float2 pc = p[i];
    pc.x = fmaf(b, pc.x, zc.x);
    pc.y = fmaf(b, pc.y, zc.y);
    p[i] = pc;
  }
}

__global__ void k_copy2(const float2* __restrict__ a, float2* __restrict__ b, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = a[i];
}

// z = N(r) with the input scale taken from the solver state
int fcg_precondition(sqcg_nn* nn, int gate, cudaStream_t s) {
  sqcg_ctx* ctx = nn->ctx;
  const int Vh = ctx->g.Vh, grid = blas_grid(ctx);
  k_norm_gated<<<grid, kRedThreads, 0, s>>>(ctx->r32, Vh, ctx->st, ctx->partials);
  SQCG_CUDA_TRY(cudaGetLastError());
  SQCG_TRY(launch_finish(ctx, grid, FIN_NN_SCALE, gate, s));
  return nn_forward_infer(nn, ctx->r32, nn->z, &ctx->st->nn_s, ctx->st, gate, s);
}

// One flexible-CG iteration in three parts: head (A p, <p,Ap>, alpha; x, r update, |r|^2), the
// FP64 reliable update (fcg_reliable), tail (z = N(r), beta, p = z + beta p).
int fcg_head(sqcg_nn* nn, void* x, cudaStream_t cs) {
  sqcg_ctx* ctx = nn->ctx;
  const int Vh = ctx->g.Vh, grid = blas_grid(ctx);
  DslashLaunch L = {};
  L.out_parity = 1; L.prec = L.out_prec = SQCG_F32; L.epi = EPI_PLAIN; L.in = ctx->p32; L.out = ctx->tmp32;
  L.gate = GATE_ITER;
  SQCG_TRY(launch_dslash(ctx, L, cs));
  L = DslashLaunch{};
  L.out_parity = 0; L.prec = L.out_prec = SQCG_F32; L.epi = EPI_NORMAL_DOT; L.in = ctx->tmp32; L.out = ctx->Ap32;
  L.y = ctx->p32; L.sigma_dev = &ctx->st->sigma; L.gate = GATE_ITER; L.fin = FIN_FCG_PAP;
  SQCG_TRY(launch_dslash(ctx, L, cs));
  k_fcg_update<<<grid, kRedThreads, 0, cs>>>((double2*)x, ctx->r32, nn->r_old, ctx->p32, ctx->Ap32, Vh, ctx->st,
                                             ctx->partials);
  SQCG_CUDA_TRY(cudaGetLastError());
  return launch_finish(ctx, grid, FIN_UPDATE, GATE_ITER, cs);
}

int fcg_tail(sqcg_nn* nn, cudaStream_t cs) {
  sqcg_ctx* ctx = nn->ctx;
  const int Vh = ctx->g.Vh, grid = blas_grid(ctx);
  SQCG_TRY(fcg_precondition(nn, GATE_ITER, cs));
  k_fcg_dots<<<grid, kRedThreads, 0, cs>>>(nn->z, ctx->r32, nn->r_old, Vh, ctx->st, ctx->partials);
  SQCG_CUDA_TRY(cudaGetLastError());
  SQCG_TRY(launch_finish2(ctx, grid, FIN_FCG_BETA, GATE_ITER, cs));
  k_fcg_xpay<<<grid, kRedThreads, 0, cs>>>(nn->z, ctx->p32, 3 * Vh, ctx->st);
  SQCG_CUDA_TRY(cudaGetLastError());
  return SQCG_OK;
}

int fcg_body(sqcg_nn* nn, void* x, cudaStream_t cs, cudaGraph_t* ifbody, cudaGraphConditionalHandle* hif_out) {
  SQCG_TRY(fcg_head(nn, x, cs));
  // IF node: reliable update r = b - A x (FP64)
  cudaStreamCaptureStatus status;
  cudaGraph_t capg = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  cudaGraphConditionalHandle hif = 0;
  SQCG_CUDA_TRY(cudaStreamGetCaptureInfo(cs, &status, nullptr, &capg, &deps, nullptr, &ndeps));
  SQCG_CUDA_TRY(cudaGraphConditionalHandleCreate(&hif, capg, 0, 0));
  cudaGraphNodeParams ip = {};
  ip.type = cudaGraphNodeTypeConditional;
  ip.conditional.handle = hif;
  ip.conditional.type = cudaGraphCondTypeIf;
  ip.conditional.size = 1;
  cudaGraphNode_t inode;
  SQCG_CUDA_TRY(cudaGraphAddNode(&inode, capg, deps, nullptr, ndeps, &ip));
  SQCG_CUDA_TRY(cudaStreamUpdateCaptureDependencies(cs, &inode, nullptr, 1, cudaStreamSetCaptureDependencies));
  *ifbody = ip.conditional.phGraph_out[0];
  *hif_out = hif;
  SQCG_TRY(fcg_tail(nn, cs));
  return launch_loop_control(nn->ctx, cs);
}

int fcg_reliable(sqcg_nn* nn, const void* b, void* x, cudaStream_t cs) {
  sqcg_ctx* ctx = nn->ctx;
  DslashLaunch L = {};
  L.out_parity = 1; L.prec = L.out_prec = SQCG_F64; L.epi = EPI_PLAIN; L.in = x; L.out = ctx->tmp64;
  L.gate = GATE_UPDATE;
  SQCG_TRY(launch_dslash(ctx, L, cs));
  L = DslashLaunch{};
  L.out_parity = 0; L.prec = SQCG_F64; L.out_prec = SQCG_F32; L.epi = EPI_TRUE_RESID; L.in = ctx->tmp64;
  L.out = ctx->r32; L.y = x; L.b = b; L.sigma_dev = &ctx->st->sigma; L.gate = GATE_UPDATE; L.fin = FIN_TRUE_RESID;
  return launch_dslash(ctx, L, cs);
}

int fcg_graph(sqcg_nn* nn, const void* b, void* x, cudaGraphExec_t* exec, cudaGraphConditionalHandle* hw,
              cudaGraphConditionalHandle* hif) {
  sqcg_ctx* ctx = nn->ctx;
  cudaStream_t cs = ctx->cap_stream;
  cudaGraph_t top = nullptr;
  SQCG_CUDA_TRY(cudaGraphCreate(&top, 0));
  int rc = SQCG_OK;
  cudaGraph_t ifbody = nullptr;
  do {
    if (cudaGraphConditionalHandleCreate(hw, top, 1, cudaGraphCondAssignDefault) != cudaSuccess) { rc = SQCG_ERR_CUDA; break; }
    cudaGraphNodeParams wp = {};
    wp.type = cudaGraphNodeTypeConditional;
    wp.conditional.handle = *hw;
    wp.conditional.type = cudaGraphCondTypeWhile;
    wp.conditional.size = 1;
    cudaGraphNode_t wnode;
    if (cudaGraphAddNode(&wnode, top, nullptr, nullptr, 0, &wp) != cudaSuccess) { rc = SQCG_ERR_CUDA; break; }
    if (cudaStreamBeginCaptureToGraph(cs, wp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal) != cudaSuccess) { rc = SQCG_ERR_CUDA; break; }
    rc = fcg_body(nn, x, cs, &ifbody, hif);
    cudaGraph_t got = nullptr;
    cudaError_t e = cudaStreamEndCapture(cs, &got);
    if (rc != SQCG_OK) break;
    if (e != cudaSuccess) { rc = SQCG_ERR_CUDA; break; }
    if (cudaStreamBeginCaptureToGraph(cs, ifbody, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) != cudaSuccess) { rc = SQCG_ERR_CUDA; break; }
    rc = fcg_reliable(nn, b, x, cs);
    e = cudaStreamEndCapture(cs, &got);
    if (rc != SQCG_OK) break;
    if (e != cudaSuccess) { rc = SQCG_ERR_CUDA; break; }
    if (cudaGraphInstantiate(exec, top, 0) != cudaSuccess) { rc = SQCG_ERR_CUDA; break; }
  } while (0);
  if (rc == SQCG_ERR_CUDA) sqcg_set_last_cuda_error(cudaGetLastError(), "flexible CG graph", __FILE__, __LINE__);
  cudaGraphDestroy(top);
  return rc;
}

// The same iterations launched one kernel at a time (SQCG_LAUNCH_MODE=eager), the host reading
// the state where the graph's conditional nodes branch, for kernel-level profilers.
int fcg_eager(sqcg_nn* nn, const void* b, void* x, cudaStream_t s) {
  sqcg_ctx* ctx = nn->ctx;
  SolverState* h = ctx->st_host;
  auto read = [&]() -> int {
    SQCG_CUDA_TRY(cudaMemcpyAsync(h, ctx->st, sizeof(SolverState), cudaMemcpyDeviceToHost, s));
    SQCG_CUDA_TRY(cudaStreamSynchronize(s));
    return SQCG_OK;
  };
  SQCG_TRY(read());
  const int limit = h->loop_limit;
  int it = 0;
  while (!h->done) {
    SQCG_TRY(fcg_head(nn, x, s));
    SQCG_TRY(read());
    if (!h->done && h->need_update) {
      SQCG_TRY(fcg_reliable(nn, b, x, s));
      SQCG_TRY(read());
    }
    if (!h->done) {
      SQCG_TRY(fcg_tail(nn, s));
      SQCG_TRY(read());
    }
    if (++it >= limit && !h->done) {  // the loop-control kernel's bound
      h->done = 1;
      h->status = SQCG_ERR_NOT_CONVERGED;
    }
  }
  h->loop_count = it;
  return SQCG_OK;
}

}  // namespace

int cg_solve_sigma(sqcg_ctx* ctx, double sigma, const void* b, void* x, double tol, int max_iter, int mode,
                   sqcg_info* info);

namespace {
// r32 = (float) r64; e32 = (float)(xs - xk)
__global__ void k_pair(const double2* r64, const double2* xs, const double2* xk, float2* r32, float2* e32, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double2 r = r64[i], a = xs[i], b = xk[i];
  r32[i] = make_float2((float)r.x, (float)r.y);
  e32[i] = make_float2((float)(a.x - b.x), (float)(a.y - b.y));
}
}  // namespace

extern "C" int sqcg_make_training_pair(sqcg_ctx* ctx, double sigma, const void* b, const void* x_k,
                                       const void* x_star, void* r_out, void* e_out) {
  if (!ctx || !b || !x_k || !x_star || !r_out || !e_out || !isfinite(sigma)) return SQCG_ERR_INVALID_ARG;
  if (!ctx->have_links) return SQCG_ERR_NO_LINKS;
  SQCG_TRY(ensure_workspace(ctx));
  cudaStream_t s = ctx->stream;
  DslashLaunch L = {};
  L.out_parity = 1; L.prec = L.out_prec = SQCG_F64; L.epi = EPI_PLAIN; L.in = x_k; L.out = ctx->tmp64;
  SQCG_TRY(launch_dslash(ctx, L, s));
  L = DslashLaunch{};
  L.out_parity = 0; L.prec = L.out_prec = SQCG_F64; L.epi = EPI_TRUE_RESID; L.in = ctx->tmp64; L.out = ctx->r64;
  L.y = x_k; L.b = b; L.sigma = sigma;
  SQCG_TRY(launch_dslash(ctx, L, s));
  const int n = 3 * ctx->g.Vh;
  k_pair<<<nn_grid(n), kThreads, 0, s>>>(ctx->r64, (const double2*)x_star, (const double2*)x_k, (float2*)r_out,
                                         (float2*)e_out, n);
  SQCG_CUDA_TRY(cudaGetLastError());
  return SQCG_OK;
}

extern "C" int sqcg_fcg_solve_nn(sqcg_ctx* ctx, sqcg_nn* nn, double mass, const void* b, void* x, double tol,
                                 int max_iter, sqcg_info* info) {
  const auto t0 = std::chrono::steady_clock::now();
  if (!ctx || !nn || nn->ctx != ctx || !b || !x || b == x || !(tol > 0) || max_iter <= 0 || !isfinite(mass))
    return SQCG_ERR_INVALID_ARG;
  if ((((uintptr_t)b) | ((uintptr_t)x)) & 15) return SQCG_ERR_INVALID_ARG;
  if (!ctx->have_links) return SQCG_ERR_NO_LINKS;
  SQCG_TRY(ensure_workspace(ctx));
  cudaStream_t s = ctx->stream;
  const int Vh = ctx->g.Vh;
  const double sigma = 4.0 * mass * mass;
  SolverState* h = ctx->st_host;
  memset(h, 0, sizeof(SolverState));
  h->sigma = sigma;
  h->stop_rr = tol * tol;
  h->delta2 = ctx->ru_delta * ctx->ru_delta;
  h->max_iter = max_iter;
  h->update_interval = ctx->ru_interval;
  h->mixed = 1;
  h->vh = Vh;
  h->status = SQCG_OK;
  SQCG_CUDA_TRY(cudaMemcpyAsync(ctx->st, h, sizeof(SolverState), cudaMemcpyHostToDevice, s));
  SQCG_TRY(launch_norm2_f64(ctx, (const double2*)b, FIN_BB, s));
  // |x0|^2: a zero initial guess has the exact initial residual r = b (no FP64 Dslash)
  SQCG_TRY(launch_norm2_f64(ctx, (const double2*)x, FIN_STORE, s));
  SQCG_CUDA_TRY(cudaMemcpyAsync(h, ctx->st, sizeof(SolverState), cudaMemcpyDeviceToHost, s));
  SQCG_CUDA_TRY(cudaStreamSynchronize(s));
  int launches = 4;
  if (h->pAp == 0.0) {
    SQCG_TRY(layout_convert(ctx, SQCG_F64, b, SQCG_F32, ctx->r32, s));
    const double v = h->bb;  // the initial-residual step of the device state, |r|^2 = |b|^2
    if (!isfinite(v)) {
      h->status = SQCG_ERR_BREAKDOWN;
      h->done = 1;
    } else {
      h->rr = h->rr_true = h->rr_max = h->rr_prev = v;
      h->iter_last_update = 0;
      if (v <= h->stop_rr) h->done = 1;
    }
    SQCG_CUDA_TRY(cudaMemcpyAsync(ctx->st, h, sizeof(SolverState), cudaMemcpyHostToDevice, s));
    launches += 1;
  } else {
    // r = b - A x0 (FP64) into r32
    DslashLaunch L = {};
    L.out_parity = 1; L.prec = L.out_prec = SQCG_F64; L.epi = EPI_PLAIN; L.in = x; L.out = ctx->tmp64;
    SQCG_TRY(launch_dslash(ctx, L, s));
    L = DslashLaunch{};
    L.out_parity = 0; L.prec = SQCG_F64; L.out_prec = SQCG_F32; L.epi = EPI_TRUE_RESID; L.in = ctx->tmp64;
    L.out = ctx->r32; L.y = x; L.b = b; L.sigma = sigma; L.fin = FIN_INIT;
    SQCG_TRY(launch_dslash(ctx, L, s));
    launches += 3;
  }
  // then z = N(r); p = z; rz = <z, r>
  SQCG_CUDA_TRY(cudaMemcpyAsync(h, ctx->st, sizeof(SolverState), cudaMemcpyDeviceToHost, s));
  SQCG_CUDA_TRY(cudaStreamSynchronize(s));
  int status = SQCG_OK, fallback = 0, iters = 0, updates = 0;
  double rel = 0.0;
  if (h->bb == 0.0) {
    SQCG_CUDA_TRY(cudaMemsetAsync(x, 0, (size_t)Vh * 3 * sizeof(double2), s));
    SQCG_CUDA_TRY(cudaStreamSynchronize(s));
  } else if (h->done) {
    status = h->status;  // x0 solves the system, or a non-finite start
    rel = sqrt(h->rr_true / h->bb);
  } else {
    // z0 = N(r0); p0 = z0; <z0, r0> (first of the two sums of k_fcg_dots)
    const int grid = blas_grid(ctx);
    SQCG_TRY(fcg_precondition(nn, GATE_ITER, s));
    k_fcg_dots<<<grid, kRedThreads, 0, s>>>(nn->z, ctx->r32, ctx->r32, Vh, ctx->st, ctx->partials);
    SQCG_CUDA_TRY(cudaGetLastError());
    SQCG_TRY(launch_finish(ctx, grid, FIN_FCG_INIT, GATE_ITER, s));
    k_copy2<<<nn_grid(3 * Vh), kThreads, 0, s>>>(nn->z, ctx->p32, 3 * Vh);
    SQCG_CUDA_TRY(cudaGetLastError());
    launches += 8;
    const char* mode = getenv("SQCG_LAUNCH_MODE");
    const bool eager = mode && strcmp(mode, "eager") == 0;
    if (!eager && (!nn->fcg_exec || nn->fcg_b != b || nn->fcg_x != x || nn->fcg_gen != ctx->links_gen)) {
      SQCG_CUDA_TRY(cudaStreamSynchronize(s));
      if (nn->fcg_exec) cudaGraphExecDestroy(nn->fcg_exec);
      nn->fcg_exec = nullptr;
      SQCG_TRY(fcg_graph(nn, b, x, &nn->fcg_exec, &nn->fcg_hw, &nn->fcg_hif));
      nn->fcg_b = b;
      nn->fcg_x = x;
      nn->fcg_gen = ctx->links_gen;
    }
    SQCG_CUDA_TRY(cudaMemcpyAsync(h, ctx->st, sizeof(SolverState), cudaMemcpyDeviceToHost, s));
    SQCG_CUDA_TRY(cudaStreamSynchronize(s));
    // no launch after a breakdown of the network output on the first residual
    cudaGraphExec_t exec = (h->done || eager) ? nullptr : nn->fcg_exec;
    h->h_while = nn->fcg_hw;
    h->h_if = nn->fcg_hif;
    h->use_if = eager ? 0 : 1;  // eager: the kernels must not touch conditional handles
    h->loop_count = 0;
    h->loop_limit = max_iter + 4;
    SQCG_CUDA_TRY(cudaMemcpyAsync(ctx->st, h, sizeof(SolverState), cudaMemcpyHostToDevice, s));
    if (eager) {
      SQCG_TRY(fcg_eager(nn, b, x, s));
    } else {
      cudaError_t e = exec ? cudaGraphLaunch(exec, s) : cudaSuccess;
      if (e == cudaSuccess) e = cudaMemcpyAsync(h, ctx->st, sizeof(SolverState), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) { sqcg_set_last_cuda_error(e, "flexible CG", __FILE__, __LINE__); return SQCG_ERR_CUDA; }
    }
    launches += h->loop_count * 14 + h->updates * 3;
    iters = h->iter;
    updates = h->updates;
    status = h->done ? h->status : SQCG_ERR_NOT_CONVERGED;
    rel = sqrt(h->rr_true / h->bb);
    if (status != SQCG_OK) {
      // plain CG takes over from the current iterate (it also judges the final answer)
      fallback = 1;
      sqcg_info ci;
      const int left = max_iter - iters > 0 ? max_iter - iters : 1;
      status = cg_solve_sigma(ctx, sigma, b, x, tol, left, SQCG_MODE_MIXED, &ci);
      if (status == SQCG_ERR_CUDA || status == SQCG_ERR_INVALID_ARG || status == SQCG_ERR_NO_MEMORY) return status;
      iters += ci.iters;
      updates += ci.reliable_updates;
      rel = ci.true_rel_resid;
      launches += ci.launches;
    }
  }
  if (info) {
    info->iters = iters;
    info->reliable_updates = updates;
    info->status = status;
    info->true_rel_resid = rel;
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    info->launches = launches;
    info->fallback = fallback;
  }
  return status;
}
