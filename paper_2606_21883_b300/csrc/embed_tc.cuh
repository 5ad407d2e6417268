// embed_tc.cuh — the FP32 walk on an embedded sphere Q S^d + b in R^n with the
// projection Q^T g of every Gaussian vector on the 5th-generation tensor cores
// (the dense contraction of the closest point Q normalize(Q^T (x - b)) + b of
// the projected chain, Sec. 2, eq. projected_chain_update).
//
// One persistent CTA of 512 threads per SM walks tiles of 128 walkers in
// lockstep: a closed embedded sphere has constant radius, so every walk of the
// tile stops at the same index.  For each Gaussian vector of a step (the
// interior samples Z_l, then the sphere sample Theta) the tile's components are
// generated in K-chunks of 64 — four threads per walker, one 16-component
// group (3 Philox blocks: two of radial words, one of 16-bit angles) each, the
// same draws as the FP32 warp walk (walkn32.cuh) — split into BF16
// hi + lo and stored into a 128-byte-swizzled K-major A tile (128 rows =
// walkers; two stages).  One elected thread issues, per 16-wide K slice, three
// tcgen05.mma kind::f16 products into one FP32 TMEM accumulator (128 x 32):
//   A_hi B_hi + A_hi B_lo + A_lo B_hi,   B = Q^T (32 x K, BF16 hi and lo),
// the two correction products refining the BF16 product to ~2^-17 relative.
// B stays resident in shared memory for the whole launch.  Chunks hand over
// through mbarriers, not CTA barriers: every warp arrives once on the stage's
// `full` barrier after its threads' stores and proxy fences, the issuing thread
// waits for it, and
// tcgen05.commit arrives on the stage's `empty` barrier, which producers wait
// on only before reusing the stage; the phase parities follow from a
// CTA-uniform chunk counter.  Warps 0..3 read their 32 TMEM lanes (walkers)
// with tcgen05.ld, 8 columns at a time, and finish the step in FP32 registers;
// each walker's state row (s, W, S) lives in shared memory.  (1024 threads at
// 64 registers measured slower on B300: the Gaussian generation, not the
// contraction or the hand-over, bounds this kernel.)  Every mbarrier wait
// is bounded; on expiry the CTA records a status bit and stops.
#pragma once
#include "dev_common.cuh"
#include "green.cuh"

namespace mpwos {
namespace tc {

constexpr int kThreads = 512;
constexpr int kM = 128;                   // walkers per tile = accumulator rows = TMEM lanes
constexpr int kTPW = kThreads / kM;       // generator threads per walker
constexpr int kUPT = 8 / kTPW;            // 16-byte units (8 components) per thread per chunk
constexpr int kN = 32;                    // accumulator columns (d + 1 <= 31, zero padded)
constexpr int kChunkK = 64;               // BF16 elements per 128-byte row
constexpr int kMaxChunks = 16;            // n <= 1024
constexpr int kBChunk = kN * 128;         // one B chunk (4 KB)
constexpr int kAHalf = kM * 128;          // one A chunk, hi or lo (16 KB)
constexpr int kBBytes = 2 * kMaxChunks * kBChunk;   // B hi + lo: 128 KB
constexpr int kABytes = 2 * 2 * kAHalf;              // 2 stages x (hi + lo): 64 KB
constexpr int kMiscBytes = 64 + 4 * kThreads + 4 * 32 * 32 + 4 * 32 + 64;
constexpr int kSStride = 37;                 // walker row: s[0..31], W (hi, lo), S (hi, lo); odd: conflict-free
constexpr int kSBytes = kM * kSStride * 4;   // 18.5 KB
static_assert(kTPW * kUPT * 8 == kChunkK && kUPT * 8 == 16, "one 16-component group per thread per chunk");
constexpr int kSmemBytes = kBBytes + kABytes + kMiscBytes + kSBytes + 1024;   // + 1 KB alignment slack
constexpr uint32_t kStatusTimeout = 1u;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t addr, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(addr), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t addr) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}" ::"r"(addr) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t addr, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(addr), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for the phase of the given parity to complete; false when about one
// second (2^31 SM cycles) passes first.
__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t parity) {
  if (mbar_try_wait(addr, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(addr, parity))
    if (clock64() - t0 > (1LL << 31)) return false;
  return true;
}

__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// D[tmem] (+)= A[smem] B[smem]^T: BF16 operands, FP32 accumulator.
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}

// 8 consecutive FP32 columns of this thread's TMEM lane (completes at tmem_wait).
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr)
               : "memory");
}
__device__ __forceinline__ void tmem_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Columns 0 .. NC-1 of this thread's TMEM lane (warps 0..3: lane = thread).
template <int NC>
__device__ __forceinline__ void tmem_row(uint32_t taddr, float (&v)[NC]) {
  static_assert(NC % 8 == 0, "whole 8-column pieces");
  uint32_t r[NC / 8][8];
  const uint32_t base = taddr + ((static_cast<uint32_t>(threadIdx.x >> 5) * 32u) << 16);
#pragma unroll
  for (int c8 = 0; c8 < NC / 8; ++c8) tmem_ld8(base + static_cast<uint32_t>(8 * c8), r[c8]);
  tmem_wait();
#pragma unroll
  for (int c8 = 0; c8 < NC / 8; ++c8)
#pragma unroll
    for (int j = 0; j < 8; ++j) v[8 * c8 + j] = __uint_as_float(r[c8][j]);
}

// Shared-memory matrix descriptor of a K-major, 128-byte-swizzled operand:
// start address, stride between 8-row groups 1024 bytes, descriptor version 1,
// swizzle mode 2 (128 B).  The leading-dimension offset is unused here.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
  uint64_t d = static_cast<uint64_t>((saddr >> 4) & 0x3FFFu);
  d |= static_cast<uint64_t>(1) << 16;
  d |= static_cast<uint64_t>(1024 >> 4) << 32;
  d |= static_cast<uint64_t>(1) << 46;
  d |= static_cast<uint64_t>(2) << 61;
  return d;
}

// Instruction descriptor of kind::f16: FP32 D, BF16 A and B, both K-major,
// N = 32 (bits 17..22 hold N/8), M = 128 (bits 24..28 hold M/16).
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((static_cast<uint32_t>(kN) >> 3) << 17) |
                            ((static_cast<uint32_t>(kM) >> 4) << 24);

// Byte offset of 16-byte unit u of row r in a 128-byte-swizzled tile.
__device__ __forceinline__ uint32_t sw128(uint32_t r, uint32_t u) { return r * 128u + ((u ^ (r & 7u)) << 4); }

// Two FP32 values rounded to BF16; `first` lands in the low half (lower address).
__device__ __forceinline__ uint32_t pack_bf16x2(float first, float second) {
  uint32_t r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(second), "f"(first));
  return r;
}
__device__ __forceinline__ float bf16_low(uint32_t packed) { return __uint_as_float(packed << 16); }
__device__ __forceinline__ float bf16_high(uint32_t packed) { return __uint_as_float(packed & 0xFFFF0000u); }

// Shared memory of both tensor-core kernels, addressed from one 1 KB-aligned
// base (the period of the 128-byte swizzle) so that only one pointer stays live.
struct Smem {
  unsigned char* base;
  __device__ __forceinline__ unsigned char* B() const { return base; }             // Q^T hi chunks, then lo
  __device__ __forceinline__ unsigned char* A() const { return base + kBBytes; }   // stage s: hi, lo
  __device__ __forceinline__ unsigned char* misc() const { return base + kBBytes + kABytes; }
  __device__ __forceinline__ uint64_t* empty() const { return reinterpret_cast<uint64_t*>(misc()); }
  __device__ __forceinline__ uint64_t* full() const { return reinterpret_cast<uint64_t*>(misc() + 16); }
  __device__ __forceinline__ uint32_t* tmem_slot() const { return reinterpret_cast<uint32_t*>(misc() + 32); }
  __device__ __forceinline__ float* consts() const { return reinterpret_cast<float*>(misc() + 40); }   // 6 floats
  __device__ __forceinline__ float* gg_part() const { return reinterpret_cast<float*>(misc() + 64); }
  __device__ __forceinline__ float* Af() const { return gg_part() + kThreads; }   // 32 x 32, zero padded
  __device__ __forceinline__ float* vf() const { return Af() + 32 * 32; }         // 32, zero padded
  __device__ __forceinline__ float* rows() const { return reinterpret_cast<float*>(misc() + kMiscBytes); }
};

// The walk's Gaussian vector v of step kk of walk (p, wi) in 16-component
// groups: group G (components 16 G .. 16 G + 15, zero past n) by
// gauss_group16, the draws of the CUDA-core walk (walkn32.cuh, gen_groups);
// returns the group's part of |g|^2.
struct PhiloxSource {
  const PhiloxKeys* K;
  Philox32Step st;
  uint32_t X;   // A0 ^ 256 v
  int n;
  __device__ __forceinline__ float operator()(int G, float (&g)[16]) const {
    if (16 * G >= n) {
#pragma unroll
      for (int q = 0; q < 16; ++q) g[q] = 0.0f;
      return 0.0f;
    }
    return gauss_group16(X, G, st, *K, n, g);
  }
};

// Row `row` of a caller-given rows x n FP32 matrix (verification primitive).
struct MatrixSource {
  const float* G;
  int64_t row, rows;
  int n;
  __device__ __forceinline__ float operator()(int grp, float (&g)[16]) const {
    float s = 0.0f;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int c = 16 * grp + q;
      g[q] = (row < rows && c < n) ? G[row * n + c] : 0.0f;
      s += g[q] * g[q];
    }
    return s;
  }
};

// Q^T g into the TMEM accumulator (row = walker) for the vector that `src`
// generates; returns |g|^2 to threads < 128.  Thread (row, part) generates
// group 4 c + part of each chunk c (components 64 c + 16 part + 0..15), the
// 16-byte units kUPT part + 0 .. kUPT - 1 of the chunk.  g is the CTA's running chunk
// count (uniform): chunk g uses stage g & 1 for the (g >> 1)-th time.  The
// caller reads TMEM (warps 0..3, warp-uniformly) and then calls tc_fence_before.
template <class Src>
__device__ __forceinline__ float project_vector(const Smem& sm, uint32_t taddr, int nchunks, const Src& src,
                                                uint32_t& g, bool& ok) {
  const int tid = threadIdx.x;
  const uint32_t row = static_cast<uint32_t>(tid & (kM - 1));
  const int part = tid / kM;
  float acc = 0.0f;
  for (int c = 0; c < nchunks; ++c) {
    const uint32_t gc = g + static_cast<uint32_t>(c), s = gc & 1u, u = gc >> 1;
    if (u >= 1 && ok) ok = mbar_wait(smem_u32(&sm.empty()[s]), (u - 1) & 1u);   // chunk gc - 2 has left the stage
    unsigned char* Ahi = sm.A() + (2 * s) * kAHalf;
    unsigned char* Alo = Ahi + kAHalf;
    float gq[16];   // the thread's group 4 c + part: components 64 c + 16 part + 0..15
    acc += src(4 * c + part, gq);
#pragma unroll
    for (int uu = 0; uu < kUPT; ++uu) {   // a 16-byte unit = 8 components
      const int unit = kUPT * part + uu;
      uint32_t hw[4], lw[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float g0 = gq[8 * uu + 2 * e], g1 = gq[8 * uu + 2 * e + 1];
        const uint32_t h01 = pack_bf16x2(g0, g1);
        hw[e] = h01;
        lw[e] = pack_bf16x2(g0 - bf16_low(h01), g1 - bf16_high(h01));
      }
      const uint32_t off = sw128(row, static_cast<uint32_t>(unit));
      *reinterpret_cast<uint4*>(Ahi + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
      *reinterpret_cast<uint4*>(Alo + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
    }
    fence_proxy_async();   // this thread's generic-proxy stores -> visible to the tensor core
    __syncwarp();
    if ((tid & 31) == 0) mbar_arrive(smem_u32(&sm.full()[s]));   // one arrival per warp
    if (tid == 0) {
      if (ok) ok = mbar_wait(smem_u32(&sm.full()[s]), u & 1u);
      tc_fence_after();
      const uint32_t a_hi = smem_u32(Ahi), a_lo = smem_u32(Alo);
      const uint32_t b_hi = smem_u32(sm.B() + c * kBChunk), b_lo = smem_u32(sm.B() + (kMaxChunks + c) * kBChunk);
#pragma unroll
      for (int k4 = 0; k4 < kChunkK / 16; ++k4) {   // 16 BF16 = 32 bytes per K slice
        const uint32_t ko = static_cast<uint32_t>(k4 * 32);
        mma_bf16(taddr, desc_sw128(a_hi + ko), desc_sw128(b_hi + ko), kIdesc, (c | k4) != 0 ? 1u : 0u);
        mma_bf16(taddr, desc_sw128(a_hi + ko), desc_sw128(b_lo + ko), kIdesc, 1u);
        mma_bf16(taddr, desc_sw128(a_lo + ko), desc_sw128(b_hi + ko), kIdesc, 1u);
      }
      mma_commit(smem_u32(&sm.empty()[s]));
    }
  }
  if (tid < kM) {   // the walkers' warps wait for the last two chunks' products
    for (int c = (nchunks >= 2 ? nchunks - 2 : 0); c < nchunks; ++c) {
      const uint32_t gc = g + static_cast<uint32_t>(c);
      if (ok) ok = mbar_wait(smem_u32(&sm.empty()[gc & 1u]), (gc >> 1) & 1u);
    }
  }
  g += static_cast<uint32_t>(nchunks);
  tc_fence_after();
  sm.gg_part()[tid] = acc;
  __syncthreads();
  float gg = 0.0f;
  if (tid < kM)
#pragma unroll
    for (int t = 0; t < kTPW; ++t) gg += sm.gg_part()[tid + t * kM];
  return gg;
}

// SPHERE_QUAD source at the point z / |z| (z with DQ components, zero padded).
template <int DQ>
__device__ __forceinline__ float sphere_quad_tc(const DevProblem& pb, const Smem& sm, const float (&z)[DQ], int D) {
  float zz = 0.0f;
#pragma unroll
  for (int j = 0; j < DQ; ++j) zz += z[j] * z[j];
  const float iz = rsqrtf(zz);
  float lin = 0.0f, quad = 0.0f;
#pragma unroll
  for (int i = 0; i < DQ; ++i) {
    lin += sm.vf()[i] * z[i];
    float Az = 0.0f;
    const float4* row = reinterpret_cast<const float4*>(sm.Af() + 32 * i);
#pragma unroll
    for (int j4 = 0; j4 < DQ / 4; ++j4) {
      const float4 a4 = row[j4];
      Az += a4.x * z[4 * j4] + a4.y * z[4 * j4 + 1] + a4.z * z[4 * j4 + 2] + a4.w * z[4 * j4 + 3];
    }
    quad += z[i] * Az;
  }
  lin *= iz;
  quad *= iz * iz;
  const float c0 = pb.f.c0_f;
  if (!pb.f.apply_op) return c0 + lin + quad;
  float tr = 0.0f;
#pragma unroll
  for (int i = 0; i < DQ; ++i) tr += sm.Af()[33 * i];
  const float dm = static_cast<float>(D - 1), sg = pb.sf.sigma, mean = tr / static_cast<float>(D);
  return sg * (c0 + mean) + (dm + sg) * lin + (2.0f * (dm + 1.0f) + sg) * (quad - mean);
}

__device__ __forceinline__ Smem smem_layout(unsigned char* raw) {
  return Smem{reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(raw) + 1023) &
                                               ~static_cast<uintptr_t>(1023))};
}

// Copy the B image into shared memory, initialise the stage barriers and
// allocate the 32-column TMEM accumulator (warp 0); all threads call this.
__device__ __forceinline__ uint32_t tc_begin(const Smem& sm, const uint4* bimg) {
  const int tid = threadIdx.x;
  uint4* dst = reinterpret_cast<uint4*>(sm.B());
  for (int q = tid; q < kBBytes / 16; q += kThreads) dst[q] = bimg[q];
  if (tid == 0) {
    mbar_init(smem_u32(&sm.empty()[0]), 1);
    mbar_init(smem_u32(&sm.empty()[1]), 1);
    mbar_init(smem_u32(&sm.full()[0]), kThreads / 32);
    mbar_init(smem_u32(&sm.full()[1]), kThreads / 32);
    fence_mbar_init();
  }
  if ((tid >> 5) == 0) {
    tmem_alloc(smem_u32(sm.tmem_slot()), 32);
    tmem_relinquish();
  }
  fence_proxy_async();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  return *sm.tmem_slot();
}

// Release TMEM; after a wait that ran out, first let the products of the last
// chunk of each stage land (bounded) and record the status.  g: chunks issued.
__device__ __forceinline__ void tc_end(const Smem& sm, uint32_t taddr, bool ok, uint32_t g, unsigned* status) {
  const int tid = threadIdx.x;
  if (!ok && tid == 0) {
    for (uint32_t back = 1; back <= 2 && back <= g; ++back) {
      const uint32_t gc = g - back;
      mbar_wait(smem_u32(&sm.empty()[gc & 1u]), (gc >> 1) & 1u);
    }
    atomicOr(status, kStatusTimeout);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if ((tid >> 5) == 0) tmem_dealloc(taddr, 32);
}

template <int DQ>
__global__ void __launch_bounds__(kThreads, 1) embed_tc_kernel(const DevProblem pb) {
  extern __shared__ unsigned char smem_raw[];
  const Smem sm = smem_layout(smem_raw);
  const int tid = threadIdx.x;
  const int n = pb.n, D = pb.d + 1;
  const int nchunks = (n + kChunkK - 1) / kChunkK;
  for (int q = tid; q < 32 * 32; q += kThreads) {
    const int i = q >> 5, j = q & 31;
    sm.Af()[q] = (i < D && j < D) ? pb.f.Af[i * D + j] : 0.0f;
  }
  if (tid < 32) sm.vf()[tid] = tid < D ? pb.f.vf[tid] : 0.0f;
  // closed manifold of constant curvature: one radius and one weight pair
  const float r = pb.sf.theta * pb.sf.rho_geo;
  const float a = pb.sf.sqrt_sigma * r;
  if (tid == 0) {
    F2 c2, om2;
    if (!pb.em1_fp64) {
      weights_from_em1(em1_poly32(pb, 0.25f * a * a), pb.sf.inv_sigma, c2, om2);
    } else {
      const double ad = static_cast<double>(a);
      const double em1 = em1_series(0.5 * static_cast<double>(n - 2), 0.25 * (ad * ad));
      const double cc = 1.0 / (1.0 + em1);
      c2 = f2_from_double(cc);
      om2 = f2_from_double(one_minus_c(em1, cc) / pb.sigma);
    }
    const F2 tau = f2_from_double(pb.tau_w);
    float* cs = sm.consts();
    cs[0] = c2.hi; cs[1] = c2.lo; cs[2] = om2.hi; cs[3] = om2.lo; cs[4] = tau.hi; cs[5] = tau.lo;
  }
  const uint32_t taddr = tc_begin(sm, pb.tc_bimg);   // also makes the stores above visible

  const PhiloxKeys& K = pb.keys;
  const int nv = pb.n_v;
  const int max_steps = static_cast<int>(pb.max_steps);
  const int64_t tiles = (pb.wk_w1 - pb.wk_w0 + kM - 1) / kM;
  uint32_t gchunk = 0;
  bool ok = true;
  float* row = sm.rows() + (tid & (kM - 1)) * kSStride;   // s[0..31], W, S of this walker (threads < kM)

  for (int64_t tile = blockIdx.x; tile < tiles && ok; tile += gridDim.x) {
    const int64_t w = pb.wk_w0 + tile * kM + (tid & (kM - 1));
    const bool active = w < pb.wk_w1;
    uint32_t p = 0, wi = 0;
    if (active) {
      const WalkId id = walk_id(pb, w);
      p = id.p;
      wi = id.i;
    }
    const Philox32Walk pw = philox32_walk(wi, K);
    if (tid < kM) {
#pragma unroll
      for (int j = 0; j < DQ; ++j)
        row[j] = (active && j < D) ? static_cast<float>(pb.s0[static_cast<size_t>(p) * D + j]) : 0.0f;
      row[32] = 1.0f; row[33] = 0.0f;   // W
      row[34] = 0.0f; row[35] = 0.0f;   // S
    }
    bool running = active && tid < kM;
    int flag = 0;
    int k = 0;       // the tile's step index: uniform over the CTA (it keys every draw)
    int kstop = 0;   // this walker's stopping index K
    for (;;) {
      if (running) {
        const float* cs = sm.consts();
        const float wh = row[32], wl = row[33];
        if (wh < cs[4] || (wh == cs[4] && wl < cs[5])) {
          running = false;
        } else if (k >= max_steps) {
          running = false;
          flag = 1;
        }
        kstop = k;
      }
      if (!__syncthreads_or(running)) break;
      const Philox32Step st = philox32_step(pw, static_cast<uint32_t>(k), p, K);
      // interior samples Z_l = s + r t_l g_l / |g_l| and the source average F
      float F = 0.0f;
      for (int l = 0; l < nv; ++l) {
        float t = 0.0f;
        if (tid < kM) {
          const U4 bu = philox32_block(pw.A0 ^ static_cast<uint32_t>(256 * (1 + nv) + (l >> 2)), st, K);
          const int s4 = l & 3;
          const float U = u23(s4 == 0 ? bu.x : (s4 == 1 ? bu.y : (s4 == 2 ? bu.z : bu.w)));
          t = fminf(fmaxf(table_lookup32(pb, a, U), 0.0f), 1.0f);
        }
        const PhiloxSource src{&K, st, pw.A0 ^ static_cast<uint32_t>(256 * (1 + l)), n};
        const float gg = project_vector(sm, taddr, nchunks, src, gchunk, ok);
        if (tid < kM) {
          float z[DQ];
          tmem_row<DQ>(taddr, z);
          const float zs = (r * t) * rsqrtf(fmaxf(gg, 1e-30f));
#pragma unroll
          for (int j = 0; j < DQ; ++j) z[j] = row[j] + zs * z[j];
          F += sphere_quad_tc<DQ>(pb, sm, z, D);
        }
        tc_fence_before();
      }
      if (nv > 1) F /= static_cast<float>(nv);
      // Theta = s + r g / |g|, then the closest point: s = Theta / |Theta|
      const PhiloxSource src{&K, st, pw.A0, n};
      const float gg = project_vector(sm, taddr, nchunks, src, gchunk, ok);
      if (tid < kM) {
        float th[DQ];
        tmem_row<DQ>(taddr, th);
        if (running) {
          const float sc = r * rsqrtf(fmaxf(gg, 1e-30f));
          float tt = 0.0f;
#pragma unroll
          for (int j = 0; j < DQ; ++j) {
            th[j] = row[j] + sc * th[j];
            tt += th[j] * th[j];
          }
          const float it = rsqrtf(tt);
#pragma unroll
          for (int j = 0; j < DQ; ++j) row[j] = th[j] * it;
          const float* cs = sm.consts();
          const F2 W{row[32], row[33]}, S{row[34], row[35]};
          const F2 S2 = f2_add(S, f2_mul_f(f2_mul(W, F2{cs[2], cs[3]}), F));
          const F2 W2 = f2_mul(W, F2{cs[0], cs[1]});
          row[32] = W2.hi; row[33] = W2.lo; row[34] = S2.hi; row[35] = S2.lo;
        }
      }
      tc_fence_before();
      ++k;
      if (!__syncthreads_and(ok)) {
        ok = false;
        break;
      }
    }
    if (tid < kM && active && ok) {
      const int64_t o = walk_id(pb, w).o;
      pb.S_out[o] = f2_to_double(F2{row[34], row[35]});
      pb.K_out[o] = kstop;
      pb.flag_out[o] = flag;
    }
  }
  tc_end(sm, taddr, ok, gchunk, pb.dev_status);
}

// Verification primitive: out[row][0..31] = (Q^T g_row) and gg[row] = |g_row|^2
// for the rows of a rows x n FP32 matrix G, through the walk's contraction path.
__global__ void __launch_bounds__(kThreads, 1) tc_project_kernel(const uint4* bimg, const float* G, int64_t rows,
                                                                 int n, float* out, float* gg_out, unsigned* status) {
  extern __shared__ unsigned char smem_raw[];
  const Smem sm = smem_layout(smem_raw);
  const int tid = threadIdx.x;
  const int nchunks = (n + kChunkK - 1) / kChunkK;
  const uint32_t taddr = tc_begin(sm, bimg);
  uint32_t gchunk = 0;
  bool ok = true;
  const int64_t tiles = (rows + kM - 1) / kM;
  for (int64_t tile = blockIdx.x; tile < tiles && ok; tile += gridDim.x) {
    const int64_t row = tile * kM + (tid & (kM - 1));
    const MatrixSource src{G, row, rows, n};
    const float gg = project_vector(sm, taddr, nchunks, src, gchunk, ok);
    if (tid < kM) {
      float q[32];
      tmem_row<32>(taddr, q);
      if (row < rows) {
#pragma unroll
        for (int j = 0; j < 32; ++j) out[row * 32 + j] = q[j];
        gg_out[row] = gg;
      }
    }
    tc_fence_before();
    if (!__syncthreads_and(ok)) ok = false;
  }
  tc_end(sm, taddr, ok, gchunk, status);
}

}  // namespace tc
}  // namespace mpwos
