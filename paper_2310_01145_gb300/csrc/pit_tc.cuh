// FP64-accurate block-level matrix products on the fifth-generation tensor cores (tcgen05).
//
// GB300 executes FP64 at 2 FMA per clock per SM; its bf16 tensor cores at about 3.5k FMA per
// clock per SM.  The large-state solver's dense D x D products (Section 3.1.2's operators on
// square-root factors) are computed here on the tensor cores without giving up FP64 accuracy, by
// the error-free splitting of Ozaki, Ogita, Oishi and Rump (2012) in its fixed-point form:
//
//  * every row i of op(A) is scaled by 2^-ea_i and every column j of op(B) by 2^-eb_j, powers of
//    two chosen so that the scaled entries lie in (-1, 1); each scaled entry is truncated to a
//    63-bit signed fixed-point number a = sum_s d_s 2^(7 (8 - s)) of NDIG = 9 signed 7-bit
//    digits, |d_s| <= 127, and digit s is stored as the bf16 d_s 2^(-7 s) (exact);
//  * the digit matrices are multiplied on the tensor cores (kind::f16, bf16 inputs, FP32
//    accumulators in tensor memory).  The pairs (s, t) of one weight group g = s + t contribute
//    integer multiples of 2^(-7 g) below 2^(14 - 7 g); groups g = 0 .. 5 (at most 6 pairs) each
//    have their own accumulator and are accumulated over at most KACC = 160 terms, so every
//    partial sum is an integer multiple of 2^(-7 g) below 6 * 160 * 127^2 2^(-7 g) < 2^(24 - 7 g)
//    and their FP32 accumulation is exact; groups 6 .. 8 share one accumulator, at most 2^-38 of
//    the leading group, whose accumulation on the tensor cores keeps about 21 bits (measured:
//    the addends span many binades and the hardware does not round them like sequential FP32
//    additions); groups g >= 9 are not formed (45 of the 81 digit pairs are multiplied);
//  * the accumulators are read out of tensor memory every KACC terms, combined exactly in 64-bit
//    integers (groups 0-3 and the rest), converted to FP64 once per window and output and scaled
//    back by 2^(ea_i + eb_j); a product with K > KACC adds its windows in FP64.
//
// The error of an output is below about 2^-58 K max_l |op(A)_il| max_l |op(B)_lj| (truncation of
// the digits, the shared accumulator and the dropped groups): entries down to about 2^-6 of their
// row's or column's largest keep the FP64 product's precision.  Non-finite inputs make the outputs
// of their row or column NaN; subnormal inputs count as zero.
//
// Operands are staged in shared memory in the canonical K-major layout without swizzling: 8-row
// x 16-byte core matrices, stored contiguously (row r of a core matrix at byte 16 r), adjacent
// along K at LBO = 128 bytes and adjacent along M/N at SBO = (KC / 8) * 128 bytes.  One thread
// issues the MMAs and commits them to an mbarrier; every wait on it is bounded (it gives up after
// 4 s of wall time and records the failure, and later products of the block are skipped).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace pit {
namespace tc {

constexpr int NDIG = 9;              // 7-bit digits per value (63-bit fixed point)
constexpr int GMAX = 8;              // largest weight group g = s + t formed (45 digit pairs)
constexpr int NEXACT = 6;            // groups 0 .. 5 exact, one accumulator each
constexpr int NACC = NEXACT + 1;     // + one accumulator shared by groups 6 .. GMAX
constexpr int TM = 128;              // rows of an MMA tile (TMEM lanes)
constexpr int TN = 64;               // columns of an MMA tile
constexpr int KC = 32;               // K staged in shared memory per chunk
constexpr int KACC = 160;            // K accumulated in TMEM between readouts (exactness bound)
constexpr int TMEM_COLS = 512;       // >= NACC * TN, a power of two
constexpr int A_SLICE = TM * KC * 2; // bytes of one digit slice of an A chunk (8 KB)
constexpr int B_SLICE = TN * KC * 2; // bytes of one digit slice of a B chunk (4 KB)
constexpr int LBO = 128, SBO = (KC / 8) * 128;
constexpr unsigned kTcWaitNs = 4000000000u;   // 4 s
static_assert(NACC * TN <= TMEM_COLS, "accumulators exceed the tensor memory allocation");
static_assert(KACC % KC == 0 && NEXACT * KACC * 127 * 127 < (1 << 24), "exact groups must stay exact");

// Shared-memory bytes of the staging area (digit slices of one A and one B chunk).
constexpr size_t stage_bytes() { return static_cast<size_t>(NDIG) * (A_SLICE + B_SLICE); }

// ---- PTX wrappers --------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint64_t gtimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Whole warp: allocates ncols (a power of two >= 32) TMEM columns, address written to *dst.
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// Generic-proxy writes to shared memory made visible to the tensor cores (async proxy).
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// D[tmem] (+)= A[smem desc] * B[smem desc]^T, bf16 inputs, FP32 accumulate; M = 128.
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// Arrive on the mbarrier once every MMA this thread issued before has completed.
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}
// 8 consecutive 32-bit columns of this thread's TMEM lane (warp w reads lanes 32 (w % 4) + laneid).
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                 "=r"(r[7])
               : "r"(taddr)
               : "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Shared-memory matrix descriptor: start address, leading (K) and stride (M/N) byte offsets,
// descriptor version 1, base offset 0, no swizzling.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4) | (static_cast<uint64_t>(lbo >> 4) << 16) |
         (static_cast<uint64_t>(sbo >> 4) << 32) | (1ull << 46);
}
// Instruction descriptor of kind::f16: FP32 accumulator, bf16 A and B, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
         (static_cast<uint32_t>(M >> 4) << 24);
}


// ---- per-block state -------------------------------------------------------------------------------
// Lives in static shared memory (one instance per thread block of every kernel that uses the
// products); the digit slices are staged in a caller-provided shared-memory area of
// stage_bytes() that may alias other scratch (nothing in it outlives a product).
struct TcShared {
  uint64_t bar;     // mbarrier: completes when every thread and the MMA commit have arrived
  uint32_t tmem;    // base address of the block's tensor memory
  uint32_t fail;    // a wait gave up: later products of the block are skipped (outputs NaN)
  uint32_t where;   // 1 + the number of chunks committed before the wait that gave up
  uint32_t count;   // chunks committed
  int ea[TM];       // scale exponents of the rows of the current op(A) tile
  int eb[TN];       // scale exponents of the columns of the current op(B) tile
};

__device__ __forceinline__ TcShared& tc_state() {
  __shared__ TcShared s;
  return s;
}

struct TcCtx {
  unsigned char* stage;   // stage_bytes() of shared memory, 128-byte aligned
  unsigned* gstatus;      // global status word: bit kTcTimeoutBit set when a wait gives up
  uint64_t wait_ns;       // wall-time limit of one wait
};

constexpr unsigned kTcTimeoutBit = 4u;

// All threads of the block, once per kernel before the first product: allocates the block's
// tensor memory and initialises the mbarrier (expected arrivals: every thread + the commit).
// Pair with tc_teardown on every path out of the kernel.
__device__ __forceinline__ void tc_setup() {
  TcShared& ts = tc_state();
  if (threadIdx.x < 32) {
    tmem_alloc(&ts.tmem, TMEM_COLS);
    tmem_relinquish();
  }
  if (threadIdx.x == 32) {
    mbar_init(&ts.bar, blockDim.x + 1);
    ts.fail = 0;
    ts.where = 0;
    ts.count = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
}

// All threads, once at the end of the kernel: frees the tensor memory.
__device__ __forceinline__ void tc_teardown() {
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (threadIdx.x < 32) tmem_dealloc(tc_state().tmem, TMEM_COLS);
}

// All threads: arrives on the mbarrier and waits for the phase to complete (every thread and
// the commit of the MMAs issued since the previous wait).  Bounded by wait_ns of wall time; a
// thread that gives up marks the block failed and sets the status bit.
__device__ __forceinline__ void tc_wait(const TcCtx& c) {
  TcShared& ts = tc_state();
  const uint32_t bar = smem_u32(&ts.bar);
  uint64_t state;
  asm volatile("mbarrier.arrive.shared::cta.b64 %0, [%1];" : "=l"(state) : "r"(bar) : "memory");
  auto test = [&]() -> bool {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "l"(state)
        : "memory");
    return ok != 0;
  };
  if (!test()) {
    const uint64_t t0 = gtimer_ns();
    uint32_t polls = 0;
    while (!test()) {
      if ((++polls & 255u) == 0 && gtimer_ns() - t0 > c.wait_ns) {
        atomicExch(&ts.fail, 1u);
        atomicCAS(&ts.where, 0u, 1u + ts.count);
        if (c.gstatus) atomicOr(c.gstatus, kTcTimeoutBit);
        break;
      }
    }
  }
  tc_fence_after();
}

// ---- FP64 -> digits ------------------------------------------------------------------------------
// a * b + c on bf16 pairs (one rounding).
__device__ __forceinline__ uint32_t bf16x2_fma(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm("fma.rn.bf16x2 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}

// Biased exponent field of x (0 for zero and subnormals, 2047 for non-finite values).
__device__ __forceinline__ int bexp(double x) {
  return static_cast<int>((static_cast<unsigned long long>(__double_as_longlong(x)) >> 52) & 0x7FFu);
}

// Writes the NDIG digits of NV consecutive K values x[e] of one row, whose scale exponent (largest
// biased exponent of the row of op(A) or column of op(B)) is emax: digit s of the values, as the
// bf16 numbers d_s 2^(-7 s), goes to the 2 NV bytes at slice0 + s * slice_bytes (x[e] at byte 2 e).
template <int NV>
__device__ __forceinline__ void split_store(const double (&x)[NV], int emax, unsigned char* slice0,
                                            int slice_bytes) {
  static_assert(NV == 4 || NV == 8, "4 or 8 values (8 or 16 bytes per digit slice)");
  unsigned long long mag[NV];
  uint32_t sgn[NV];
#pragma unroll
  for (int e = 0; e < NV; ++e) {
    const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x[e]));
    const int E = static_cast<int>((b >> 52) & 0x7FFu);
    const unsigned long long M = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int sh = E - emax + 10;   // <= 10: |x| 2^(1085 - emax) < 2^63
    unsigned long long m = 0;
    if (E != 0 && emax != 2047) m = sh >= 0 ? (M << sh) : (sh > -64 ? (M >> (-sh)) : 0ull);
    mag[e] = m;
    sgn[e] = static_cast<uint32_t>(b >> 63) << 15;
  }
#pragma unroll
  for (int sl = 0; sl < NDIG; ++sl) {
    const int shift = 7 * (NDIG - 1 - sl);
    // bf16 pairs 2^(-7 sl) and -128 2^(-7 sl) (exact powers of two)
    const uint32_t sc = static_cast<uint32_t>(127 - 7 * sl) << 7;
    const uint32_t nb = 0x8000u | (static_cast<uint32_t>(134 - 7 * sl) << 7);
    uint32_t w[NV / 2];
#pragma unroll
    for (int q = 0; q < NV / 2; ++q) {
      const uint32_t d0 = static_cast<uint32_t>(mag[2 * q] >> shift) & 127u;
      const uint32_t d1 = static_cast<uint32_t>(mag[2 * q + 1] >> shift) & 127u;
      // 0x4300 | d is the bf16 128 + d exactly; (128 + d) 2^(-7 sl) - 128 2^(-7 sl) is the bf16
      // d 2^(-7 sl) exactly: two digits per packed fma
      w[q] = bf16x2_fma(0x43004300u | d0 | (d1 << 16), sc | (sc << 16), nb | (nb << 16)) |
             sgn[2 * q] | (sgn[2 * q + 1] << 16);
    }
    if constexpr (NV == 8)
      *reinterpret_cast<uint4*>(slice0 + sl * slice_bytes) = make_uint4(w[0], w[1], w[2], w[3]);
    else
      *reinterpret_cast<uint2*>(slice0 + sl * slice_bytes) = make_uint2(w[0], w[1]);
  }
}

// Writes zero digits (NDIG slices of 2 NV bytes) for a quarter row outside the operand.
template <int NV>
__device__ __forceinline__ void zero_store(unsigned char* slice0, int slice_bytes) {
#pragma unroll
  for (int sl = 0; sl < NDIG; ++sl) {
    if constexpr (NV == 8) *reinterpret_cast<uint4*>(slice0 + sl * slice_bytes) = make_uint4(0, 0, 0, 0);
    else *reinterpret_cast<uint2*>(slice0 + sl * slice_bytes) = make_uint2(0, 0);
  }
}

// Byte offset of row r, K-octet o of a digit slice in the canonical no-swizzle K-major layout.
__device__ __forceinline__ uint32_t core_off(int r, int o) {
  return static_cast<uint32_t>((r >> 3) * SBO + o * LBO + (r & 7) * 16);
}

// An FP32 number holding an integer of magnitude below 2^62, as a 64-bit integer, with integer
// operations only (the hardware conversion runs on the FP64 pipe).
__device__ __forceinline__ long long f2ll_exact(float x) {
  const uint32_t b = __float_as_uint(x);
  const int E = static_cast<int>((b >> 23) & 0xFFu);
  const long long M = static_cast<long long>((b & 0x7FFFFFu) | 0x800000u);
  const long long m = E >= 150 ? (M << (E - 150)) : (E >= 127 ? (M >> (150 - E)) : 0ll);
  return (b >> 31) ? -m : m;
}

// ---- MMA issue and readout --------------------------------------------------------------------------
// One thread: the MMAs of one staged chunk (45 digit pairs x 2 K-steps of 16) into the
// accumulators (group g -> accumulator min(g, NEXACT)), then a commit.  first: the chunk opens a
// readout window (each accumulator's first MMA of the chunk resets it).  Fully unrolled: every
// descriptor is a base plus a compile-time offset (the start-address field counts 16 bytes).
template <int G, int S>
__device__ __forceinline__ void tc_issue_pair(uint64_t ad0, uint64_t bd0, uint32_t tm, bool first) {
  constexpr int T = G - S;
  constexpr int ACC = G < NEXACT ? G : NEXACT;
  // the accumulator's first MMA of the chunk: pair S == 0 of group G (exact groups) or the
  // first pair of group NEXACT (shared accumulator)
  constexpr bool opens = (G < NEXACT && S == 0) || (G == NEXACT && S == 0);
  constexpr uint32_t id = idesc_bf16(TM, TN);
#pragma unroll
  for (int ks = 0; ks < KC / 16; ++ks) {
    const uint64_t ad = ad0 + static_cast<uint64_t>((S * A_SLICE + ks * 2 * LBO) >> 4);
    const uint64_t bd = bd0 + static_cast<uint64_t>((T * B_SLICE + ks * 2 * LBO) >> 4);
    mma_bf16(tm + ACC * TN, ad, bd, id, (opens && ks == 0 && first) ? 0u : 1u);
  }
}
template <int G, int S>
__device__ __forceinline__ void tc_issue_group(uint64_t ad0, uint64_t bd0, uint32_t tm, bool first) {
  if constexpr (S <= G) {
    if constexpr (S < NDIG && G - S < NDIG) tc_issue_pair<G, S>(ad0, bd0, tm, first);
    tc_issue_group<G, S + 1>(ad0, bd0, tm, first);
  }
}
template <int G>
__device__ __forceinline__ void tc_issue_groups(uint64_t ad0, uint64_t bd0, uint32_t tm, bool first) {
  if constexpr (G <= GMAX) {
    tc_issue_group<G, 0>(ad0, bd0, tm, first);
    tc_issue_groups<G + 1>(ad0, bd0, tm, first);
  }
}
static __device__ __noinline__ void tc_issue_chunk(const TcCtx c, bool first) {
  const uint32_t sa = smem_u32(c.stage), sb = sa + NDIG * A_SLICE;
  tc_issue_groups<0>(smem_desc(sa, LBO, SBO), smem_desc(sb, LBO, SBO), tc_state().tmem, first);
  mma_commit(&tc_state().bar);
}

// All threads: 8 outputs of the accumulators as 64-bit integers S with shifts x, the scaled
// product being S 2^(ea + eb - 2114 + x).  Thread (warp w, lane l) reads tile row 32 (w % 4) + l
// and tile columns 16 (w / 4) + 8 h .. + 7.  The groups 0-3 (multiples of 2^-21 below 2^25) and
// the rest (multiples of 2^-56 below 2^-3; the shared accumulator rounded to an integer) are each
// summed exactly in 64-bit integers, hi and lo; S = hi 2^(35 - x) + floor(lo 2^-x) with the
// smallest x >= 0 that keeps |S| < 2^63, so that the dropped bits are below 2^-60 of |S|.
__device__ __forceinline__ void tc_read8(int h, long long (&out)[8], int (&sh)[8]) {
  const int warp = threadIdx.x >> 5;
  const uint32_t base = tc_state().tmem + (static_cast<uint32_t>(32 * (warp & 3)) << 16) +
                        static_cast<uint32_t>(16 * (warp >> 2) + 8 * h);
  float v[NACC][8];
#pragma unroll
  for (int a = 0; a < NACC; ++a) tmem_ld8(base + a * TN, v[a]);
  tmem_wait_ld();
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    long long hi = 0;
#pragma unroll
    for (int a = 0; a < 4; ++a) hi += f2ll_exact(v[a][e] * 2097152.0f);           // 2^21
    const long long lo = f2ll_exact(v[4][e] * 72057594037927936.0f) +              // 2^56
                         f2ll_exact(v[5][e] * 72057594037927936.0f) +
                         f2ll_exact(v[6][e] * 72057594037927936.0f);
    const long long ahi = hi < 0 ? -hi : hi;
    const int x = max(0, 64 - __clzll(ahi) - 27);   // |hi| < 2^(27 + x)
    out[e] = hi * (1ll << (35 - x)) + (lo >> x);
    sh[e] = x;
  }
}

// S 2^x as an FP64 number (one conversion; the scaling adds to the exponent field when the
// result is a normal number, else ldexp).
__device__ __forceinline__ double tc_scaled(long long S, int x) {
  const double v = __ll2double_rn(S);
  const long long b = __double_as_longlong(v);
  const int E = static_cast<int>((b >> 52) & 0x7FF);
  if (E == 0) return v;   // zero
  const int En = E + x;
  if (En >= 1 && En <= 2046) return __longlong_as_double(b + (static_cast<long long>(x) << 52));
  return ldexp(v, x);
}

__device__ __forceinline__ double tc_nan() { return __longlong_as_double(0x7FF8000000000000ll); }

// ---- block GEMM ------------------------------------------------------------------------------------
// The product op(A)[m x k] op(B)[k x n] in FP64 accuracy on the tensor cores, with the operands
// read through getA(i, l) = op(A)[i][l] and getB(l, j) = op(B)[l][j] and the result delivered
// through put(i, j, v, first): once per output and window of KACC terms, v the window's part of
// (op(A) op(B))[i][j] and first true for the first window (NaN for every window after a wait
// gave up; v = 0 once when k == 0).  The getters may read any memory the block can see; put must
// only write memory the getters do not read.  All NT = 512 threads of the block; inputs
// visible on entry, everything put wrote visible to the block on return.
template <class GA, class GB, class PUT>
__device__ __noinline__ void cta_dgemm_f(const TcCtx c, int m, int n, int k, GA opA, GB opB, PUT put) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  TcShared& ts = tc_state();
  int* ea = ts.ea;
  int* eb = ts.eb;
  const int nchunks = (k + KC - 1) / KC;
  // staging roles, in quarter rows of a chunk (4 consecutive K values): A quarters tid and
  // tid + 512 (rows tid / 8 and 64 + tid / 8), B quarter tid (row tid / 8)
  static_assert(TM * KC / 4 == 2 * 512 && TN * KC / 4 == 512, "staging roles assume 512 threads");
  const int rq = tid >> 3, oq = (tid >> 1) & 3, uq = tid & 1;
  const int ra0 = rq, ra1 = rq + 64, rb = rq;
  const uint32_t qoff = 8 * uq;
  // output roles: tile row orow, tile columns ocol .. ocol + 15
  const int orow = 32 * (warp & 3) + lane, ocol = 16 * (warp >> 2);
  for (int i0 = 0; i0 < m; i0 += TM) {
    __syncthreads();   // ea of the previous row tile no longer read
    {  // row tid / 4, every fourth K value from tid % 4, eight loads in flight
      const int r = tid >> 2, part = tid & 3, i = i0 + r;
      int e = 0;
      if (i < m) {
        int l = part;
        for (; l + 28 < k; l += 32) {
          double v[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) v[u] = opA(i, l + 4 * u);
#pragma unroll
          for (int u = 0; u < 8; ++u) e = max(e, bexp(v[u]));
        }
        for (; l < k; l += 4) e = max(e, bexp(opA(i, l)));
      }
      e = max(e, __shfl_xor_sync(0xffffffffu, e, 1));
      e = max(e, __shfl_xor_sync(0xffffffffu, e, 2));
      if (part == 0) ea[r] = e;
    }
    const int ia0 = i0 + ra0, ia1 = i0 + ra1;
    for (int j0 = 0; j0 < n; j0 += TN) {
      {  // column tid / 8, every eighth K value from tid % 8, eight loads in flight
        const int r = tid >> 3, part = tid & 7, j = j0 + r;
        int e = 0;
        if (j < n) {
          int l = part;
          for (; l + 56 < k; l += 64) {
            double v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = opB(l + 8 * u, j);
#pragma unroll
            for (int u = 0; u < 8; ++u) e = max(e, bexp(v[u]));
          }
          for (; l < k; l += 8) e = max(e, bexp(opB(l, j)));
        }
        e = max(e, __shfl_xor_sync(0xffffffffu, e, 1));
        e = max(e, __shfl_xor_sync(0xffffffffu, e, 2));
        e = max(e, __shfl_xor_sync(0xffffffffu, e, 4));
        if (part == 0) eb[r] = e;
      }
      __syncthreads();
      const int jb = j0 + rb;
      // a single K chunk: the A digits staged for the first column tile serve every column tile
      const bool a_resident = nchunks == 1 && j0 > 0;
      double xa0[4], xa1[4], xb[4];
      auto load = [&](int kc0) {
        const int l0 = kc0 + 8 * oq + 4 * uq;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          if (!a_resident) {
            xa0[e] = (ia0 < m && l0 + e < k) ? opA(ia0, l0 + e) : 0.0;
            xa1[e] = (ia1 < m && l0 + e < k) ? opA(ia1, l0 + e) : 0.0;
          }
          xb[e] = (jb < n && l0 + e < k) ? opB(l0 + e, jb) : 0.0;
        }
      };
      if (nchunks > 0) load(0);
      for (int ch = 0; ch < nchunks; ++ch) {
        const int kc0 = ch * KC;
        const bool kin = kc0 + 8 * oq + 4 * uq < k;
        if (!a_resident) {
          if (ia0 < m && kin) split_store<4>(xa0, ea[ra0], c.stage + core_off(ra0, oq) + qoff, A_SLICE);
          else zero_store<4>(c.stage + core_off(ra0, oq) + qoff, A_SLICE);
          if (ia1 < m && kin) split_store<4>(xa1, ea[ra1], c.stage + core_off(ra1, oq) + qoff, A_SLICE);
          else zero_store<4>(c.stage + core_off(ra1, oq) + qoff, A_SLICE);
        }
        if (jb < n && kin) split_store<4>(xb, eb[rb], c.stage + NDIG * A_SLICE + core_off(rb, oq) + qoff, B_SLICE);
        else zero_store<4>(c.stage + NDIG * A_SLICE + core_off(rb, oq) + qoff, B_SLICE);
        fence_proxy_async_smem();
        tc_fence_before();
        __syncthreads();
        const bool failed = ts.fail != 0;
        if (!failed && tid == 0) {
          tc_fence_after();
          tc_issue_chunk(c, (kc0 % KACC) == 0);
          ts.count += 1;
        }
        if (ch + 1 < nchunks) load(kc0 + KC);   // in flight while the tensor cores run
        if (failed) continue;
        tc_wait(c);
        if ((kc0 + KC) % KACC != 0 && ch + 1 < nchunks) continue;
        // readout of a window: C = beta C + alpha W (first window), C += alpha W (later ones)
        const bool first_window = kc0 < KACC;
        const int i = i0 + orow;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          long long v[8];
          int vx[8];
          tc_read8(h, v, vx);
          if (i >= m) continue;
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const int jj = ocol + 8 * h + e, j = j0 + jj;
            if (j >= n) continue;
            const int s2 = ea[orow] + eb[jj];
            const double val = (ea[orow] == 2047 || eb[jj] == 2047) ? tc_nan()
                                                                    : tc_scaled(v[e], s2 - 2114 + vx[e]);
            put(i, j, val, first_window);
          }
        }
        tc_fence_before();
      }
      __syncthreads();
      if (ts.fail != 0 || nchunks == 0) {   // a wait gave up (NaN), or k == 0 (a zero product)
        const double v = ts.fail != 0 ? tc_nan() : 0.0;
        const int i = i0 + orow;
        if (i < m) {
          for (int jj = ocol; jj < ocol + 16; ++jj) {
            const int j = j0 + jj;
            if (j < n) put(i, j, v, true);
          }
        }
      }
      __syncthreads();   // eb and the staging area are reused by the next column tile
    }
  }
}

// C[m x n] = alpha op(A)[m x k] op(B)[k x n] + beta C in FP64 accuracy on the tensor cores.
// op(A)[i][l] = TA ? A[l][i] : A[i][l]; op(B)[l][j] = TB ? B[j][l] : B[l][j].  beta == 0 does
// not read C; C must not alias A or B.  All NT = 512 threads of the block; inputs visible on
// entry, outputs visible to the block on return.  A block whose wait gave up writes NaN.
template <bool TA, bool TB>
__device__ void cta_dgemm(const TcCtx& c, int m, int n, int k, double alpha, const double* A, int lda,
                          const double* B, int ldb, double beta, double* C, int ldc) {
  const bool alpha_m1 = alpha == -1.0, alpha_1 = alpha == 1.0;
  const bool beta_0 = beta == 0.0, beta_1 = beta == 1.0;
  cta_dgemm_f(
      c, m, n, k,
      [=](int i, int l) -> double {
        return TA ? A[static_cast<size_t>(l) * lda + i] : A[static_cast<size_t>(i) * lda + l];
      },
      [=](int l, int j) -> double {
        return TB ? B[static_cast<size_t>(j) * ldb + l] : B[static_cast<size_t>(l) * ldb + j];
      },
      [=](int i, int j, double v, bool first) {
        if (alpha_m1) v = -v;
        else if (!alpha_1) v *= alpha;
        double* cp = C + static_cast<size_t>(i) * ldc + j;
        if (!first || beta_1) *cp += v;
        else if (beta_0) *cp = v;
        else *cp = fma(beta, *cp, v);
      });
}

}  // namespace tc
}  // namespace pit
