// Tall-skinny products of the BMG cycle on the 5th-generation tensor cores (tcgen05),
// with float64-class accuracy from exact BF16 digit slices.
//
//   Gram      G = X^T Y        X, Y: [n][ld] blocks, contraction over the n rows
//             (the Rayleigh-Ritz block matrices X^T A X, X^T M X of Sec. 4.1)
//   expand    U = Z + X Yx     X: [n][ld], Yx: k x k, contraction over k
//             (Ritz vectors in V_{h1} + span X: U = Q Y_c + X Y_x)
//
// GB300 retires float64 at about 1/64 of its float32 rate, while its tensor cores
// multiply BF16 at petaflop rates.  Both products are therefore formed from integer
// digits, in the manner of Ozaki, Ogita, Oishi & Rump (2012, "Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication"), but with the exactness carried by integer arithmetic:
//
//  1. Scaling.  Every value x of a scaling group (Gram: one column of X or Y over a
//     window of 256 rows; expand: one row of X over its k values, one column of Yx)
//     with group exponent E (the largest biased exponent in the group, so that
//     |x| < 2^(E - bias + 1)) is turned into the integer V = round(x 2^(F - E + bias
//     - 1)), |V| <= 2^F, F = 7 S - 1.
//  2. Digits.  V = sum_{s=1..S} d_s 2^(7 (S - s)) with balanced digits
//     d_s in [-64, 64]; every digit is a BF16 value exactly.
//  3. Products.  For every digit pair (s, t) with s + t <= T the tensor cores
//     accumulate sum_r d_s(x_r) d_t(y_r) in float32 in tensor memory; pairs with
//     the same diagonal s + t share an accumulator.  A diagonal holds at most 8
//     pairs over at most 256 terms of magnitude <= 2^12, so every partial sum is an
//     integer of magnitude <= 2^23 and the float32 accumulation is exact.
//  4. Combination.  The diagonals of a window are read back (tcgen05.ld), turned
//     into int32 exactly, and combined with shifts into one int64 per output
//     element; windows are added in int64 after aligning their exponents.  Only the
//     last step, int64 -> float64 times a power of two, uses float64 arithmetic.
//
// Error: dropping the pairs s + t > T and rounding V leave an error below about
// (T - 1) 2^(-7 (T - 1)) K max|x| max|y| per window of K terms: 2^-53 for float64
// blocks (S = 8, T = 9, 36 pairs), 2^-33 for float32 blocks (S = 5, T = 6,
// 15 pairs), where the data themselves carry 2^-24.
//
// Kernel structure (one CTA per SM: 192 KB of shared memory, up to 512 TMEM
// columns).  Operand digits are written by all threads into shared memory in the
// no-swizzle K-major core-matrix layout (8 rows x 16 bytes per core matrix), two
// stages; one thread issues tcgen05.mma (kind::f16, BF16 x BF16 -> FP32, M = 128,
// N = 64) and commits to an mbarrier per stage, so that the digits of the next
// 32-row sub-chunk are formed while the tensor cores work on the current one.  Every
// wait is bounded (about 2 s of clock); on expiry the kernel raises *err, waits a
// bounded time more, frees its tensor memory and returns.
#include <algorithm>
#include <cstring>

#include "common.cuh"

namespace bmg {
namespace {

constexpr int kWorkers = 512;             // 16 warps forming digits and reading TMEM back; warps w,
                                         // w+4, w+8, w+12 share TMEM lanes
constexpr int kTcThreads = kWorkers + 32; // and one warp that issues the MMAs
constexpr int kMmaWarp = kWorkers / 32;
constexpr int kKsub = 32;                // K rows per sub-chunk (two MMA K-steps of 16)
constexpr int kWindow = 256;             // K rows per exact accumulation window (Gram)
constexpr int kNB = 64;                  // output columns per CTA (N of the MMA)
constexpr int kBeta = 7;                 // digit width
constexpr long long kWaitCycles = 4000000000LL;   // ~2 s at 2 GHz

// Digit layout of one operand (rows x kKsub, BF16, K-major, no swizzle).
constexpr int kAPlane = 128 * kKsub * 2;  // bytes per digit plane of the 128-row operand
constexpr int kBPlane = kNB * kKsub * 2;  // bytes per digit plane of the 64-row operand

__host__ __device__ constexpr int stage_bytes(int S) { return S * (kAPlane + kBPlane); }

// byte offset of the 8-element K-group starting at (row, k0) (k0 % 8 == 0)
__device__ __forceinline__ int cm_off(int row, int k0) {
  return (row >> 3) * (kKsub * 16) + (k0 >> 3) * 128 + (row & 7) * 16;
}

// ------------------------------------------------------------ PTX wrappers ----
__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor (tcgen05): start address, leading byte offset
// (distance of the two K-adjacent core matrices), stride byte offset (distance of
// 8-row groups), descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((addr & 0x3FFFF) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}
// Instruction descriptor, kind::f16: BF16 A and B (K-major), FP32 D, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(id), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
               : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Waits for the completion of the phase with the given parity; false after `limit`
// clocks without it (kWaitCycles, about 2 s, except in the timeout self-test).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long limit) {
  const long long t0 = clock64();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(su32(bar)), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > limit) return false;
  }
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// int32 of a float32 holding an integer (exact: |value| <= 2^23 here)
__device__ __forceinline__ int f2i_exact(uint32_t bits) { return __float2int_rn(__uint_as_float(bits)); }

// ------------------------------------------------------------ digits ----------
template <typename T> struct Fmt;
// emax: the biased exponent of Inf and NaN.  A group holding one has that group
// exponent, and every output it contributes to is NaN.
template <> struct Fmt<double> {
  static constexpr int bias = 1023, p = 53, emax = 2047;   // p: significand bits incl. the hidden one
  __device__ static int expo(double x) { return (int)((__double_as_longlong(x) >> 52) & 0x7FF); }
  // V = round(x 2^(F - E + bias - 1)) for |x| < 2^(E - bias + 1)
  __device__ static long long fixed(double x, int E, int F) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7FF);
    if (e == 0 || e == emax) return 0;   // zero, subnormal (below every digit), or not finite
    const long long m = (long long)((b & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull);
    const int sh = e - E + F - p;
    long long v;
    if (sh >= 0) v = m << sh;
    else if (sh < -60) v = 0;
    else v = (m + (1ll << (-sh - 1))) >> (-sh);
    return (b >> 63) ? -v : v;
  }
};
template <> struct Fmt<float> {
  static constexpr int bias = 127, p = 24, emax = 255;
  __device__ static int expo(float x) { return (int)((__float_as_uint(x) >> 23) & 0xFF); }
  __device__ static long long fixed(float x, int E, int F) {
    const uint32_t b = __float_as_uint(x);
    const int e = (int)((b >> 23) & 0xFF);
    if (e == 0 || e == emax) return 0;
    const long long m = (long long)((b & 0x7FFFFFu) | 0x800000u);
    const int sh = e - E + F - p;
    long long v;
    if (sh >= 0) v = m << sh;
    else if (sh < -40) v = 0;
    else v = (m + (1ll << (-sh - 1))) >> (-sh);
    return (b >> 31) ? -v : v;
  }
};

// 64 sum_{s < S-1} 2^(7 s): the bias 64 in each of the S - 1 lower digits
__host__ __device__ constexpr long long digit_bias(int S) {
  long long b = 0;
  for (int s = 0; s + 1 < S; ++s) b = b * 128 + 64;
  return b;
}

// float32 value u - 64 of a 7-bit field u = (x >> sh) & 127 (exact): the field is put
// into the low mantissa bits of 1.5 2^23 (one LOP3) and 1.5 2^23 + 64 subtracted.
__device__ __forceinline__ float biased_digit(uint32_t x_shifted) {
  return __uint_as_float((x_shifted & 127u) | 0x4B400000u) - 12582976.0f;
}
// two float32 integers of at most 8 significant bits as one BF16 pair (exact): the
// top halves of their bit patterns, the first in the low half
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  return __byte_perm(__float_as_uint(lo), __float_as_uint(hi), 0x7632);
}

// Balanced base-2^7 digits of the 8 integers v[0..7] (|v| <= 2^(7 S - 1)): writes S
// planes of 16 bytes (8 BF16 values each) at dst + s * plane_stride, s = 0 the most
// significant digit.  With the bias B = 64 sum_{s < S-1} 2^(7 s), w = v + B holds
// the digits d_s + 64 in [0, 127] as its ordinary base-2^7 digits below the top one,
// and the top digit d_{S-1} = w >> 7 (S - 1) (arithmetic): the digits of the
// division-by-2^7 recursion d = ((v + 64) mod 2^7) - 64, v <- (v - d) / 2^7, each
// read by one shift of w.
template <int S, int NV>
__device__ __forceinline__ void store_digits(const long long (&v)[NV], unsigned char* dst, int plane_stride) {
  static_assert(NV == 4 || NV == 8, "4 or 8 values (8 or 16 bytes per plane)");
  constexpr long long B = digit_bias(S);
  uint32_t packed[S][NV / 2];
#pragma unroll
  for (int q = 0; q < NV; q += 2) {
    const long long w0 = v[q] + B, w1 = v[q + 1] + B;
    const uint32_t l0 = (uint32_t)w0, h0 = (uint32_t)((unsigned long long)w0 >> 32);
    const uint32_t l1 = (uint32_t)w1, h1 = (uint32_t)((unsigned long long)w1 >> 32);
#pragma unroll
    for (int s = 0; s < S - 1; ++s) {   // s-th least significant digit -> plane S - 1 - s
      const int sh = kBeta * s;
      const uint32_t x0 = sh < 32 ? __funnelshift_r(l0, h0, sh) : (h0 >> (sh - 32));
      const uint32_t x1 = sh < 32 ? __funnelshift_r(l1, h1, sh) : (h1 >> (sh - 32));
      packed[S - 1 - s][q >> 1] = pack_bf16(biased_digit(x0), biased_digit(x1));
    }
    constexpr int top = kBeta * (S - 1);
    const int t0 = (int)(w0 >> top), t1 = (int)(w1 >> top);
    packed[0][q >> 1] = pack_bf16(__int_as_float(0x4B400000 + t0) - 12582912.0f,
                                  __int_as_float(0x4B400000 + t1) - 12582912.0f);
  }
#pragma unroll
  for (int s = 0; s < S; ++s) {
    if constexpr (NV == 8)
      *reinterpret_cast<uint4*>(dst + s * plane_stride) = make_uint4(packed[s][0], packed[s][1], packed[s][2], packed[s][3]);
    else
      *reinterpret_cast<uint2*>(dst + s * plane_stride) = make_uint2(packed[s][0], packed[s][1]);
  }
}

// byte offset of the 4 K-elements starting at (row, k4) (k4 % 4 == 0): the low or
// high half of a core-matrix row
__device__ __forceinline__ int quad_off(int row, int k4) { return cm_off(row, k4 & ~7) + (k4 & 4) * 2; }

// Issues the MMAs of one sub-chunk: every digit pair (s, t) with s + t <= T into the
// accumulator of its diagonal (columns (s + t - 2) * kNB of the allocation).
// first: the sub-chunk opens an accumulation window (the first MMA into each
// diagonal overwrites it).
template <int S, int T>
__device__ __forceinline__ void issue_mmas(uint32_t tmem, uint32_t sA, uint32_t sB, bool first) {
  constexpr uint32_t id = idesc_bf16(128, kNB);
#pragma unroll
  for (int dg = 2; dg <= T; ++dg) {
    const int s0 = dg - S > 1 ? dg - S : 1;
    const int s1 = dg - 1 < S ? dg - 1 : S;
#pragma unroll
    for (int s = s0; s <= s1; ++s) {
      const int t = dg - s;
#pragma unroll
      for (int ks = 0; ks < kKsub / 16; ++ks) {
        const uint64_t ad = sdesc(sA + (s - 1) * kAPlane + ks * 256, 128, kKsub * 16);
        const uint64_t bd = sdesc(sB + (t - 1) * kBPlane + ks * 256, 128, kKsub * 16);
        const uint32_t acc = (first && s == s0 && ks == 0) ? 0u : 1u;
        mma_bf16(tmem + (uint32_t)((dg - 2) * kNB), ad, bd, id, acc);
      }
    }
  }
}

// Exact combination of the diagonals of one output element into two int64 words:
//   lo = sum_{dg = T-3..T} A_dg 2^((T - dg) beta),  hi = sum_{dg = 2..T-4} A_dg 2^((T - 4 - dg) beta),
//   sum_dg A_dg 2^((T - dg) beta) = hi 2^(4 beta) + lo,
// each word below 2^44 in magnitude for |A_dg| <= 2^23 (no bit is dropped).
constexpr int kLoShift = 4 * kBeta;
__device__ __forceinline__ long long sra(long long x, int sh) { return sh >= 63 ? (x < 0 ? -1 : 0) : (x >> sh); }

// 4 consecutive TMEM columns of this warp's 32 lanes.
__device__ __forceinline__ void tmem_ld4(uint32_t addr, uint32_t (&v)[4]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3])
               : "r"(addr));
}

// Reads the T-1 diagonals of 4 output columns of this thread's TMEM lane and
// combines them exactly into (hi, lo) word pairs.
template <int T>
__device__ __forceinline__ void read_window(uint32_t taddr, long long (&hi)[4], long long (&lo)[4]) {
  uint32_t v[T - 1][4];
#pragma unroll
  for (int dg = 2; dg <= T; ++dg) tmem_ld4(taddr + (uint32_t)((dg - 2) * kNB), v[dg - 2]);
  tmem_wait_ld();
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    long long h = 0, l = 0;
#pragma unroll
    for (int dg = 2; dg <= T; ++dg) {
      const long long a = f2i_exact(v[dg - 2][q]);
      if (dg >= T - 3) l += a << ((T - dg) * kBeta);
      else h += a << ((T - 4 - dg) * kBeta);
    }
    hi[q] = h;
    lo[q] = l;
  }
}

// (hi 2^28 + lo) / 2^sh, rounded down, as a new (hi, lo) pair (lo not normalised).
__device__ __forceinline__ void pair_sra(long long& hi, long long& lo, int sh) {
  if (sh <= 0) return;
  if (sh >= kLoShift) {
    lo = sra(hi, sh - kLoShift) + sra(lo, sh);
    hi = 0;
  } else {
    const long long q = hi >> sh;
    lo = sra(lo, sh) + ((hi - (q << sh)) << (kLoShift - sh));
    hi = q;
  }
}

// The same value hi 2^28 + lo with lo reduced into [0, 2^28), so that it fits an int32.
__device__ __forceinline__ void pair_norm(long long& hi, long long& lo) {
  hi += lo >> kLoShift;
  lo &= (1ll << kLoShift) - 1;
}

// v 2^e for a float64 v, by a power-of-two factor when 2^e is a normal number
__device__ __forceinline__ double scale2(double v, int e) {
  if (e >= -1022 && e <= 1023) return v * __longlong_as_double((long long)(e + 1023) << 52);
  return ldexp(v, e);
}
__device__ __forceinline__ double pair_value(long long hi, long long lo, int e) {
  return scale2(fma((double)hi, 268435456.0, (double)lo), e);   // 2^28
}

// exponent offset of the product value: x y = 2^(Ex + Gy + off) (hi 2^28 + lo)
template <typename TA, typename TB, int S, int T>
__host__ __device__ constexpr int value_offset() {
  return -Fmt<TA>::bias - Fmt<TB>::bias + 2 - 2 * (kBeta * S - 1) + (2 * S - T) * kBeta;
}

// Output value of the expansion: Z + (hi 2^28 + lo) 2^e (0 + Z outside the k columns).
template <typename TI> struct Epi;
template <> struct Epi<double> {
  __device__ static double out(long long hi, long long lo, bool in, int e, const double* z) {
    double v = in ? pair_value(hi, lo, e) : 0.0;
    return z ? v + *z : v;
  }
};
template <> struct Epi<float> {
  // float32 digits (T = 6): hi holds one diagonal (< 2^22), so hi 2^28 + lo < 2^51
  __device__ static float out(long long hi, long long lo, bool in, int e, const float* z) {
    float v = 0.f;
    if (in) {
      v = (float)((hi << kLoShift) + lo);
      if (e >= -126 && e <= 127) v *= __int_as_float((e + 127) << 23);
      else v = ldexpf(v, e);
    }
    return z ? v + *z : v;
  }
};

// Launch controls: the limit of every bounded wait, and (timeout self-test only) an
// MMA warp that issues nothing, so that the workers' waits for commits expire.
struct TcCtl {
  long long wait_cycles;
  int no_mma;
};

struct TcShared {
  long long wait_limit;
  int no_mma;
  uint64_t bar[2];    // stage b free again: the commit of its MMAs (one arrival)
  uint64_t full[2];   // stage b holds digits: one arrival per worker warp
  uint32_t tmem_slot;
  int abort_flag;
  int exA[128];     // exponents of the 128 A rows (Gram: columns of X; expand: rows of X)
  int exB[kNB];     // exponents of the kNB B rows (Gram: columns of Y; expand: columns of Yx)
  int gR[kNB], gW[kNB], gRun[kNB];
};

template <int S>
__device__ __forceinline__ unsigned char* stage_ptr(unsigned char* smem, int b) {
  return smem + b * stage_bytes(S);
}

// TMEM columns: one kNB-wide accumulator per diagonal, rounded up to a power of two.
template <int T>
__host__ __device__ constexpr uint32_t tmem_cols() {
  return (T - 1) * kNB <= 32 ? 32 : (T - 1) * kNB <= 64 ? 64 : (T - 1) * kNB <= 128 ? 128 : (T - 1) * kNB <= 256 ? 256 : 512;
}

// barrier of the worker warps only (the MMA warp does not take part)
__device__ __forceinline__ void workers_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kWorkers) : "memory"); }

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(su32(bar)) : "memory");
}

template <int T>
__device__ __forceinline__ void tc_setup(TcShared& sh, unsigned char* smem, int bytes, const TcCtl& ctl) {
  const int tid = threadIdx.x;
  for (int q = tid; q < bytes / 16; q += blockDim.x) reinterpret_cast<uint4*>(smem)[q] = make_uint4(0, 0, 0, 0);
  if (tid == 0) {
    sh.wait_limit = ctl.wait_cycles;
    sh.no_mma = ctl.no_mma;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&sh.bar[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&sh.bar[1])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&sh.full[0])), "n"(kWorkers / 32));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&sh.full[1])), "n"(kWorkers / 32));
    sh.abort_flag = 0;
  }
  if ((tid >> 5) == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&sh.tmem_slot)),
                 "r"(tmem_cols<T>()));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_async_smem();
  fence_before();
  __syncthreads();
  fence_after();
}

// End of a tensor-core kernel, reached by every thread.  The issuing thread first
// waits (bounded) for the last commit of each stage, so that no MMA is in flight when
// the tensor memory is freed (after a timed-out wait the MMAs may still run).
template <int T>
__device__ __forceinline__ void tc_teardown(TcShared& sh, int issued, int* err) {
  if (threadIdx.x == kWorkers) {
    for (int b = 0; b < 2; ++b) {
      const int uses = (issued - b + 1) / 2;   // commits made on stage b
      if (uses > 0 && !mbar_wait(&sh.bar[b], (uint32_t)((uses - 1) & 1), sh.wait_limit)) atomicExch(&sh.abort_flag, 1);
    }
  }
  fence_before();
  __syncthreads();
  if ((threadIdx.x >> 5) == 0) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(sh.tmem_slot), "r"(tmem_cols<T>()));
  }
  if (sh.abort_flag && threadIdx.x == 0) atomicExch(err, 1);
}

// Waits (every worker) for the commit of sub-chunk gi; raises the shared abort flag
// on expiry.  Workers read the flag only right after a worker barrier, so that they
// leave their loops together.
__device__ __forceinline__ void wait_sub(TcShared& sh, int gi) {
  if (!mbar_wait(&sh.bar[gi & 1], (uint32_t)((gi >> 1) & 1), sh.wait_limit)) atomicExch(&sh.abort_flag, 1);
}

// The MMA warp's part for sub-chunk g (sc: its index in the accumulation window):
// lane 0 waits for the workers' digits of stage g & 1, issues the MMAs and commits
// them to the stage's free barrier.  Returns false (warp-uniform) when the wait expired.
template <int S, int T>
__device__ __forceinline__ bool mma_step(TcShared& sh, unsigned char* smem, uint32_t tmem, int g, int sc) {
  const int lane = threadIdx.x & 31;
  const int b = g & 1;
  int ok = 1;
  if (lane == 0) ok = mbar_wait(&sh.full[b], (uint32_t)((g >> 1) & 1), sh.wait_limit) ? 1 : 0;
  ok = __shfl_sync(0xffffffffu, ok, 0);
  if (!ok) {
    if (lane == 0) atomicExch(&sh.abort_flag, 1);
    return false;
  }
  if (lane == 0 && !sh.no_mma) {
    fence_after();
    const uint32_t sA = su32(stage_ptr<S>(smem, b));
    issue_mmas<S, T>(tmem, sA, sA + S * kAPlane, sc == 0);
    mma_commit(&sh.bar[b]);
  }
  __syncwarp();
  return true;
}

// A worker warp hands stage b to the MMA warp: every lane's digit stores made visible
// to the tensor cores' (async) proxy, then one arrival for the warp.
__device__ __forceinline__ void hand_over(TcShared& sh, int b) {
  fence_async_smem();
  __syncwarp();
  if ((threadIdx.x & 31) == 0) mbar_arrive(&sh.full[b]);
}

// ------------------------------------------------------------ Gram kernel -----
// blockIdx.x: row part [r0, r1); blockIdx.y: block of kNB columns of Y.
// partial[part][i * k + j] = (X[r0:r1, i])^T Y[r0:r1, j] for i < k and j in the block.
// Warps 0-15 form the digits of each 32-row sub-chunk (three 4-value quads per thread:
// two of X, one of Y) and read the window sums back; warp 16 issues the MMAs.
template <typename TI, int S, int T>
__global__ void __launch_bounds__(kTcThreads, 1)
gram_tc_kernel(const TI* __restrict__ X, const TI* __restrict__ Y, int n, int k, int ld, int rows_per_part,
               double* __restrict__ partial, int* err, TcCtl ctl) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ TcShared sh;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int jb = blockIdx.y * kNB;
  const int r0 = blockIdx.x * rows_per_part;
  const int r1 = min(n, r0 + rows_per_part);
  constexpr int F = kBeta * S - 1;
  tc_setup<T>(sh, smem, 2 * stage_bytes(S), ctl);
  const uint32_t tmem = sh.tmem_slot;
  if (warp == kMmaWarp) {
    int g = 0;
    bool ok = true;
    for (int w0 = r0; w0 < r1 && ok; w0 += kWindow) {
      const int nsub = (min(r1, w0 + kWindow) - w0 + kKsub - 1) / kKsub;
      for (int sc = 0; sc < nsub && ok; ++sc) {
        ok = mma_step<S, T>(sh, smem, tmem, g, sc);
        if (ok) ++g;
      }
    }
    tc_teardown<T>(sh, sh.no_mma ? 0 : g, err);
    return;
  }
  if (tid < kNB) sh.gRun[tid] = 0;
  // readback ownership: TMEM lane i = row of the output block, 16 columns
  const int i_out = (warp & 3) * 32 + lane;
  const int c_base = (warp >> 2) * 16;
  const uint32_t tlane = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)c_base;
  // running sums of the 16 outputs of this thread: Rh 2^28 + Rl, Rl in [0, 2^28)
  long long Rh[16];
  int Rl[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) { Rh[q] = 0; Rl[q] = 0; }
  int e_run = 0;
  int g = 0;
  for (int w0 = r0; w0 < r1; w0 += kWindow) {
    const int w1 = min(r1, w0 + kWindow);
    // group exponents of the window: columns of X (A rows) and of the Y block (B rows)
    workers_sync();
    if (sh.abort_flag) break;
    if (tid < 128) sh.exA[tid] = 0;
    if (tid < kNB) sh.exB[tid] = 0;
    workers_sync();
    {
      const int c = tid & 127;
      int m = 0;
      if (c < k) {
#pragma unroll 8
        for (int r = w0 + (tid >> 7); r < w1; r += kWorkers / 128) m = max(m, Fmt<TI>::expo(X[(size_t)r * ld + c]));
      }
      if (m) atomicMax(&sh.exA[c], m);
      const int j = tid & (kNB - 1);
      int mb = 0;
      if (jb + j < k) {
#pragma unroll 8
        for (int r = w0 + (tid / kNB); r < w1; r += kWorkers / kNB) mb = max(mb, Fmt<TI>::expo(Y[(size_t)r * ld + jb + j]));
      }
      if (mb) atomicMax(&sh.exB[j], mb);
    }
    workers_sync();
    const int nsub = (w1 - w0 + kKsub - 1) / kKsub;
    for (int sc = 0; sc < nsub; ++sc, ++g) {
      const int b = g & 1;
      if (g >= 2) wait_sub(sh, g - 2);
      unsigned char* st = stage_ptr<S>(smem, b);
      const int rb = w0 + sc * kKsub;
      // X quads (column c, rows rq * 4 .. rq * 4 + 3 of the sub-chunk) and the Y quad
      // (column jb + j): the 12 values are loaded first, so that their loads are in
      // flight together
      const int c = tid & 127, j = tid & (kNB - 1), rqy = tid / kNB;
      TI xa[2][4], yb[4];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int rq = (tid >> 7) + 4 * h;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int r = rb + rq * 4 + q;
          xa[h][q] = (c < k && r < w1) ? X[(size_t)r * ld + c] : TI(0);
        }
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int r = rb + rqy * 4 + q;
        yb[q] = (jb + j < k && r < w1) ? Y[(size_t)r * ld + jb + j] : TI(0);
      }
      if (c < k) {
        const int E = sh.exA[c];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          long long v[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) v[q] = Fmt<TI>::fixed(xa[h][q], E, F);
          store_digits<S, 4>(v, st + quad_off(c, ((tid >> 7) + 4 * h) * 4), kAPlane);
        }
      }
      if (jb + j < k) {
        const int E = sh.exB[j];
        long long v[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) v[q] = Fmt<TI>::fixed(yb[q], E, F);
        store_digits<S, 4>(v, st + S * kAPlane + quad_off(j, rqy * 4), kBPlane);
      }
      hand_over(sh, b);
    }
    wait_sub(sh, g - 1);
    fence_after();
    // exponent alignment of the running sums
    if (tid < kNB) {
      const int newG = max(sh.gRun[tid], sh.exB[tid]);
      sh.gR[tid] = newG - sh.gRun[tid];
      sh.gW[tid] = newG - sh.exB[tid];
    }
    workers_sync();
    if (sh.abort_flag) break;
    const int eA = sh.exA[i_out];
    const int newE = max(e_run, eA);
    const int dR = newE - e_run, dW = newE - eA;
    e_run = newE;
#pragma unroll
    for (int ch = 0; ch < 4; ++ch) {
      long long wh[4], wl[4];
      read_window<T>(tlane + ch * 4, wh, wl);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int jj = c_base + ch * 4 + q;
        long long rh = Rh[ch * 4 + q], rl = Rl[ch * 4 + q];
        pair_sra(rh, rl, dR + sh.gR[jj]);
        pair_sra(wh[q], wl[q], dW + sh.gW[jj]);
        rh += wh[q];
        rl += wl[q];
        pair_norm(rh, rl);
        Rh[ch * 4 + q] = rh;
        Rl[ch * 4 + q] = (int)rl;
      }
    }
    fence_before();
    workers_sync();
    if (tid < kNB) sh.gRun[tid] = max(sh.gRun[tid], sh.exB[tid]);
  }
  workers_sync();
  if (!sh.abort_flag && i_out < k) {
    constexpr int off = value_offset<TI, TI, S, T>();
    double* out = partial + (size_t)blockIdx.x * k * k + (size_t)i_out * k;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int j = jb + c_base + q;
      if (j < k)
        out[j] = (e_run == Fmt<TI>::emax || sh.gRun[c_base + q] == Fmt<TI>::emax)
                     ? __longlong_as_double(0x7FF8000000000000ll)
                     : pair_value(Rh[q], (long long)Rl[q], e_run + sh.gRun[c_base + q] + off);
    }
  }
  tc_teardown<T>(sh, 0, err);
}

// ------------------------------------------------------------ expand ----------
// Digits of the B operand of the expansion, Yx (k x k, float64, row stride ldy):
// B[j][q] = Yx[q][j], per block of kNB columns j and sub-chunk of kKsub values q,
// S planes in the shared-memory layout; gexp[j] = exponent of column j.
template <int S>
__global__ void expand_prep_kernel(const double* __restrict__ Yx, int k, int ldy, int nsub,
                                   unsigned char* __restrict__ dig, int* __restrict__ gexp) {
  const int jb = blockIdx.x * kNB;
  __shared__ int ex[kNB];
  constexpr int F = kBeta * S - 1;
  const int tid = threadIdx.x;
  if (tid < kNB) {
    int m = 0;
    if (jb + tid < k)
      for (int q = 0; q < k; ++q) m = max(m, Fmt<double>::expo(Yx[(size_t)q * ldy + jb + tid]));
    ex[tid] = m;
    gexp[jb + tid] = m;
  }
  __syncthreads();
  for (int task = tid; task < nsub * 4 * kNB; task += blockDim.x) {
    const int j = task % kNB, qg = (task / kNB) % 4, sc = task / (4 * kNB);
    long long v[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int q = sc * kKsub + qg * 8 + t;
      v[t] = (jb + j < k && q < k) ? Fmt<double>::fixed(Yx[(size_t)q * ldy + jb + j], ex[j], F) : 0;
    }
    unsigned char* blk = dig + ((size_t)blockIdx.x * nsub + sc) * S * kBPlane;
    store_digits<S, 8>(v, blk + cm_off(j, qg * 8), kBPlane);
  }
}

// U[r][j] = Z[r][j] + sum_q X[r][q] Yx[q][j] for the rows of 128-row tiles and the
// columns of kNB-column blocks, tiles taken in turn by persistent CTAs.  Warps 0-15
// form the X digits of each 32-value sub-chunk (two 4-value quads per thread), copy
// the prepared Yx digits and write U; warp 16 issues the MMAs.
template <typename TI, int S, int T>
__global__ void __launch_bounds__(kTcThreads, 1)
expand_tc_kernel(const TI* __restrict__ Z, const TI* __restrict__ X, const unsigned char* __restrict__ dig,
                 const int* __restrict__ gexp, int n, int k, int ld, int nsub, int njb, TI* __restrict__ U,
                 int* err, TcCtl ctl) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ TcShared sh;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  constexpr int F = kBeta * S - 1;
  tc_setup<T>(sh, smem, 2 * stage_bytes(S), ctl);
  const uint32_t tmem = sh.tmem_slot;
  const int ntiles = (n + 127) / 128;
  if (warp == kMmaWarp) {
    int g = 0;
    bool ok = true;
    for (int task = blockIdx.x; task < ntiles * njb && ok; task += gridDim.x)
      for (int sc = 0; sc < nsub && ok; ++sc) {
        ok = mma_step<S, T>(sh, smem, tmem, g, sc);
        if (ok) ++g;
      }
    tc_teardown<T>(sh, sh.no_mma ? 0 : g, err);
    return;
  }
  const int i_out = (warp & 3) * 32 + lane;
  const int c_base = (warp >> 2) * 16;
  const uint32_t tlane = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)c_base;
  int g = 0;
  for (int task = blockIdx.x; task < ntiles * njb; task += gridDim.x) {
    const int rt = task / njb, jbi = task % njb;
    const int row0 = rt * 128, jb = jbi * kNB;
    // row exponents of the tile: 4 consecutive lanes per row, reading consecutive
    // values, reduced by shuffles
    workers_sync();
    if (sh.abort_flag) break;
    if (tid < kNB) sh.exB[tid] = gexp[jb + tid];
    {
      const int rl = tid >> 2, part = tid & 3, r = row0 + rl;
      int m = 0;
      if (r < n) {
#pragma unroll 8
        for (int q = part; q < k; q += 4) m = max(m, Fmt<TI>::expo(X[(size_t)r * ld + q]));
      }
      m = max(m, __shfl_xor_sync(0xffffffffu, m, 1));
      m = max(m, __shfl_xor_sync(0xffffffffu, m, 2));
      if (part == 0) sh.exA[rl] = m;
    }
    workers_sync();
    for (int sc = 0; sc < nsub; ++sc, ++g) {
      const int b = g & 1;
      if (g >= 2) wait_sub(sh, g - 2);
      unsigned char* st = stage_ptr<S>(smem, b);
      // X quads: row rl of the tile, values qd * 4 .. qd * 4 + 3 of the sub-chunk; 8
      // consecutive lanes cover the 32 values of one row (coalesced), both quads
      // loaded before either is converted
      const int qd = tid & 7;
      const int q0 = sc * kKsub + qd * 4;
      TI xa[2][4];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int r = row0 + (tid >> 3) + 64 * h;
#pragma unroll
        for (int q = 0; q < 4; ++q) xa[h][q] = (r < n && q0 + q < k) ? X[(size_t)r * ld + q0 + q] : TI(0);
      }
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int rl = (tid >> 3) + 64 * h;
        const int E = sh.exA[rl];
        long long v[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) v[q] = Fmt<TI>::fixed(xa[h][q], E, F);
        store_digits<S, 4>(v, st + quad_off(rl, qd * 4), kAPlane);
      }
      // Yx digits: copy of the prepared planes of this column block and sub-chunk
      {
        const uint4* src = reinterpret_cast<const uint4*>(dig + ((size_t)jbi * nsub + sc) * S * kBPlane);
        uint4* dst = reinterpret_cast<uint4*>(st + S * kAPlane);
        for (int q = tid; q < S * kBPlane / 16; q += kWorkers) dst[q] = src[q];
      }
      hand_over(sh, b);
    }
    wait_sub(sh, g - 1);
    fence_after();
    workers_sync();
    if (sh.abort_flag) break;
    const int r = row0 + i_out;
    const int eA = sh.exA[i_out];
    constexpr int off = value_offset<TI, double, S, T>();
#pragma unroll
    for (int ch = 0; ch < 4; ++ch) {
      long long wh[4], wl[4];
      read_window<T>(tlane + ch * 4, wh, wl);
      if (r < n) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int jl = c_base + ch * 4 + q, j = jb + jl;
          if (j < ld) {
            const size_t idx = (size_t)r * ld + j;
            const bool nonfinite = j < k && (eA == Fmt<TI>::emax || sh.exB[jl] == Fmt<double>::emax);
            U[idx] = nonfinite ? (TI)__longlong_as_double(0x7FF8000000000000ll)
                               : Epi<TI>::out(wh[q], wl[q], j < k, eA + sh.exB[jl] + off, Z ? Z + idx : nullptr);
          }
        }
      }
    }
    fence_before();
  }
  workers_sync();
  tc_teardown<T>(sh, 0, err);
}

template <typename TI> struct TcDigits;
template <> struct TcDigits<double> { static constexpr int S = 8, T = 9; };
template <> struct TcDigits<float> { static constexpr int S = 5, T = 6; };

int num_sms() {
  static int n = [] {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : 152;
  }();
  return n;
}

}  // namespace

int gram_tc_parts(int n, int k) {
  const int njb = (k + kNB - 1) / kNB;
  const int windows = (n + kWindow - 1) / kWindow;
  int parts = std::max(1, std::min(windows, num_sms() / njb));
  // at most 127 windows per part (headroom of the int64 window sums)
  parts = std::max(parts, (windows + 126) / 127);
  return parts;
}

size_t expand_tc_scratch_bytes(int k) {
  const int njb = (k + kNB - 1) / kNB, nsub = (k + kKsub - 1) / kKsub;
  return (size_t)njb * nsub * TcDigits<double>::S * kBPlane + sizeof(int) * njb * kNB + 256;
}

namespace {
template <typename TI>
void gram_tc_launch(const TI* X, const TI* Y, int n, int k, int ld, double* G, double* partial, int nparts,
                    int* err, cudaStream_t s, bool sym, TcCtl ctl) {
  if (k > kTcMaxK) fail(BMG_ERR_INVALID_ARG, "gram_tc: k > 128");
  constexpr int S = TcDigits<TI>::S, T = TcDigits<TI>::T;
  const int njb = (k + kNB - 1) / kNB;
  int rows = (n + nparts - 1) / nparts;
  rows = (rows + kWindow - 1) / kWindow * kWindow;
  const int parts = (n + rows - 1) / rows;
  const int smem = 2 * stage_bytes(S);
  check_cuda(cudaFuncSetAttribute(gram_tc_kernel<TI, S, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem),
             "cudaFuncSetAttribute(gram_tc_kernel)");
  prof_begin(KC_GRAM, s);
  gram_tc_kernel<TI, S, T><<<dim3(parts, njb), kTcThreads, smem, s>>>(X, Y, n, k, ld, rows, partial, err, ctl);
  check_launch("gram_tc_kernel");
  gram_reduce(partial, parts, k, G, sym, s);
  prof_end(KC_GRAM, s, 2.0 * sizeof(TI) * n * ld + 16.0 * parts * k * k + 8.0 * k * k, 2.0 * n * k * k);
}
}  // namespace

template <typename TI>
void gram_tc(const TI* X, const TI* Y, int n, int k, int ld, double* G, double* partial, int nparts, int* err,
             cudaStream_t s, bool sym) {
  gram_tc_launch<TI>(X, Y, n, k, ld, G, partial, nparts, err, s, sym, TcCtl{kWaitCycles, 0});
}

// The bounded waits of the tensor-core kernels, made to run out: a float64 Gram of a
// zero 4096 x 64 block whose MMA warp issues nothing, with waits of about 1 ms.  The
// workers' waits for the commits expire; the kernel must raise *err, free its tensor
// memory and return.  Buffers are the caller's (partial: gram_tc_parts(4096, 64) * 64^2
// doubles).
void gram_tc_timeout_selftest(const double* X, double* G, double* partial, int* err, cudaStream_t s) {
  gram_tc_launch<double>(X, X, 4096, 64, 64, G, partial, gram_tc_parts(4096, 64), err, s, true,
                         TcCtl{2000000LL, 1});
}

template <typename TI>
void expand_tc(const TI* Zf, const TI* X, const double* Yx, int n, int k, int ld, int ldy, TI* U,
               unsigned char* scratch, int* err, cudaStream_t s) {
  if (k > kTcMaxK) fail(BMG_ERR_INVALID_ARG, "expand_tc: k > 128");
  constexpr int S = TcDigits<TI>::S, T = TcDigits<TI>::T;
  const int njb = (k + kNB - 1) / kNB, nsub = (k + kKsub - 1) / kKsub;
  int* gexp = reinterpret_cast<int*>(scratch + (size_t)njb * nsub * TcDigits<double>::S * kBPlane);
  const int smem = 2 * stage_bytes(S);
  check_cuda(cudaFuncSetAttribute(expand_tc_kernel<TI, S, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem),
             "cudaFuncSetAttribute(expand_tc_kernel)");
  const int tasks = ((n + 127) / 128) * njb;
  const int grid = std::max(1, std::min(tasks, num_sms()));
  prof_begin(KC_EXPAND, s);
  expand_prep_kernel<S><<<njb, 256, 0, s>>>(Yx, k, ldy, nsub, scratch, gexp);
  check_launch("expand_prep_kernel");
  expand_tc_kernel<TI, S, T><<<grid, kTcThreads, smem, s>>>(Zf, X, scratch, gexp, n, k, ld, nsub, njb, U, err,
                                                             TcCtl{kWaitCycles, 0});
  check_launch("expand_tc_kernel");
  prof_end(KC_EXPAND, s, 3.0 * sizeof(TI) * n * ld + 8.0 * k * k, 2.0 * n * k * k);
}

template void gram_tc<double>(const double*, const double*, int, int, int, double*, double*, int, int*, cudaStream_t,
                              bool);
template void gram_tc<float>(const float*, const float*, int, int, int, double*, double*, int, int*, cudaStream_t,
                             bool);
template void expand_tc<double>(const double*, const double*, const double*, int, int, int, int, double*,
                                unsigned char*, int*, cudaStream_t);
template void expand_tc<float>(const float*, const float*, const double*, int, int, int, int, float*, unsigned char*,
                               int*, cudaStream_t);

}  // namespace bmg
