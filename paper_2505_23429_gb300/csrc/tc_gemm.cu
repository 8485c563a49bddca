// tcgen05 BF16 GEMM (TMA -> shared memory -> tcgen05.mma -> TMEM -> registers) and the
// BF16 H_eff chain built on it (sm_103a).
//
//   D[m][n] = sum_k A[m][k] * B[n][k]      A: M x K, B: N x K, both K-major BF16,
//   FP32 accumulation in tensor memory, epilogue stores BF16 or FP32 (plain or atomic).
//
// A persistent kernel (one CTA of 192 threads per SM) walks the 128 x BN output tiles
// (and their K splits): warp 0 lane 0 issues TMA loads into a STAGES-deep ring of
// 128B-swizzled tiles, warp 1 lane 0 issues tcgen05.mma (M=128, N=BN, K=16 per
// instruction) into one of two TMEM accumulators, and warps 2..5 drain the other one.
// Every mbarrier wait is bounded; a timeout raises a device error flag, every role
// leaves its loop, the in-flight copies and MMAs are waited for, TMEM is freed.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "tc_gemm.cuh"

namespace a2 {

namespace tc {

constexpr int BM = 128;
constexpr int BK = 64;              // 64 bf16 = 128 bytes = one swizzle row
constexpr uint32_t kWaitLimit = 1u << 26;

__device__ int g_tc_error = 0;     // set to a nonzero code when a bounded wait gives up

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred P;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n\t"
      "selp.b32 %0, 1, 0, P;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: returns false (and records `code`) if the phase never completes.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int code,
                                          uint32_t limit = kWaitLimit) {
  for (uint32_t it = 0; it < limit; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if (it > 64) __nanosleep(64);
  }
  atomicExch(&g_tc_error, code);
  return false;
}

__device__ __forceinline__ void tma_load_2d(const CUtensorMap* map, uint64_t* bar, void* dst,
                                            int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tma_load_3d(const CUtensorMap* map, uint64_t* bar, void* dst,
                                            int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tma_load_4d(const CUtensorMap* map, uint64_t* bar, void* dst,
                                            int x, int y, int z, int w) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(w), "r"(smem_u32(bar))
      : "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t smem_desc(const void* p) {
  const uint64_t addr = smem_u32(p);
  uint64_t d = 0;
  d |= (addr >> 4) & 0x3FFFull;            // start address
  d |= (uint64_t)1 << 16;                  // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;        // stride byte offset: 8 rows x 128 B
  d |= (uint64_t)1 << 46;                  // descriptor version for tcgen05
  d |= (uint64_t)2 << 61;                  // SWIZZLE_128B
  return d;
}

// Instruction descriptor, kind::f16: BF16 x BF16 -> FP32, both operands K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4)                     // D format F32
         | (1u << 7)                   // A format BF16
         | (1u << 10)                  // B format BF16
         | ((uint32_t)(N >> 3) << 17)  // N / 8
         | ((uint32_t)(M >> 4) << 24); // M / 16
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
        "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
        "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

enum OutKind { OUT_BF16 = 0, OUT_F32 = 1, OUT_F32_ATOMIC = 2 };

constexpr int kMaxPlanes = 8;      // BF16 planes per operand (8: the FP64 level products)
constexpr int kMaxPairs = 8;       // operand pairs accumulated into one tile

struct TcArgs {
  int M, N, K;
  int nk1, nk2;            // K blocks of the plain product and of the optional second segment
  int nbc2, n12;           // second segment: b' chunks per w1, (s1 s2) rows per a
  int kblocks_per_split;   // K blocks (of BK) in one work unit
  int splits;              // K splits (work units per output tile)
  void* C;
  long long ldc;
  int out_kind;
  int npairs;              // operand pairs accumulated into one tile (split precision)
  int pa[kMaxPairs], pb[kMaxPairs];   // A / B plane of each pair
  int tma_store;           // 1: epilogue through shared memory + TMA bulk tensor store
  long long split_ld;      // > 0: K split sp stores its own FP32 tile at C + sp * split_ld
  uint32_t wait_limit;     // iterations of every bounded wait (kWaitLimit)
  int no_loads;            // self-test only: the producer issues no copies, so the first
                           // wait of the MMA role runs out (see tc_selftest_timeout)
};

// Up to three BF16 planes per operand (a value split into high, middle and low parts).
// a2 / b2: the optional second K segment, A as a 4D view [a][w1][s12][b'] (box
// 64 x n12 x 1 x 128/n12, i.e. 128 rows (a, s12) x 64 b') and B as a 3D view
// [b][w1][b'] (box 64 x 1 x BN); both land in shared memory exactly like the 2D boxes.
struct TcMaps {
  CUtensorMap a[kMaxPlanes];
  CUtensorMap b[kMaxPlanes];
  CUtensorMap a2[3];
  CUtensorMap b2[3];
  CUtensorMap c;           // output (FP32 box 32 x 32 or BF16 box 64 x 32, 128B swizzle)
};

// Epilogue warps: 4 (one per TMEM lane quarter, each draining all BN columns), or 8 in
// the promoted mode (two per lane quarter, 128 columns each, FP32 register accumulators).
__host__ __device__ constexpr int epi_warps(bool promote) { return promote ? 8 : 4; }
__host__ __device__ constexpr int tc_threads(bool promote) { return 64 + 32 * epi_warps(promote); }

template <int BN, int STAGES, int EPI, int NBUF>
struct TcSmem {
  alignas(1024) __nv_bfloat16 a[STAGES][BM * BK];
  alignas(1024) __nv_bfloat16 b[STAGES][BN * BK];
  alignas(1024) unsigned char cbuf[EPI][NBUF][4096];      // epilogue staging buffers
  alignas(8) uint64_t full[STAGES];                // TMA -> MMA
  alignas(8) uint64_t empty[STAGES];               // MMA -> TMA
  alignas(8) uint64_t acc_full[2];                 // MMA -> epilogue (per TMEM buffer)
  alignas(8) uint64_t acc_empty[2];                // epilogue -> MMA
  alignas(8) uint64_t drain;                       // MMA completion on abort
  uint32_t tmem_base;
  int abort_flag;
};

__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, const void* src, int x,
                                             int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
          reinterpret_cast<uint64_t>(map)),
      "r"(x), "r"(y), "r"(smem_u32(src))
      : "memory");
}
__device__ __forceinline__ void tma_reduce_add_2d(const CUtensorMap* map, const void* src, int x,
                                                  int y) {
  asm volatile(
      "cp.reduce.async.bulk.tensor.2d.global.shared::cta.add.bulk_group [%0, {%1, %2}], [%3];" ::
          "l"(reinterpret_cast<uint64_t>(map)),
      "r"(x), "r"(y), "r"(smem_u32(src))
      : "memory");
}
__device__ __forceinline__ void bulk_commit() {
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_read1() {
  asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_read0() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_all() {
  asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}
__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c,
                                             uint32_t d) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c),
               "r"(d)
               : "memory");
}
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&h);
}

static_assert(sizeof(TcSmem<256, 4, 4, 2>) + 1024 <= 227 * 1024, "BN=256 ring exceeds smem");
static_assert(sizeof(TcSmem<128, 6, 4, 2>) + 1024 <= 227 * 1024, "BN=128 ring exceeds smem");
static_assert(sizeof(TcSmem<256, 4, 8, 1>) + 1024 <= 227 * 1024, "promoted ring exceeds smem");

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Bounded wait that also gives up early once another role has raised the abort flag.
__device__ __forceinline__ bool mbar_wait_or_abort(uint64_t* bar, uint32_t parity, int code,
                                                   const int* abort_flag,
                                                   uint32_t limit = kWaitLimit) {
  for (uint32_t it = 0; it < limit; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255) == 255 && *(volatile const int*)abort_flag) return false;
    if (it > 64) __nanosleep(64);
  }
  atomicExch(&g_tc_error, code);
  return false;
}

// Persistent warp-specialised GEMM.  Work unit = (128 x BN output tile, K split); CTA c
// takes units c, c + gridDim.x, ...  Warp 0 lane 0 streams (A, B) K blocks through a
// STAGES-deep ring with TMA, warp 1 lane 0 issues tcgen05.mma into one of two TMEM
// accumulators (2 x BN columns), warps 2..5 drain the other accumulator (warp w reads
// TMEM lanes 32*(w%4)..+31) and store it, so the epilogue of one unit overlaps the MMAs
// of the next.  Every wait is bounded; a timeout raises the device error flag and all
// roles leave their loops, wait (bounded) for their copies / MMAs in flight and exit.
// PROMOTE (FP32 outputs, BN = 256): the tensor cores' FP32 accumulator truncates, so
// over long reductions its error grows with the number of accumulate steps.  In this
// mode every kPromoteKB K blocks (with their operand pairs) are accumulated into a fresh
// TMEM buffer and the eight epilogue warps add the partials into IEEE FP32 registers
// (round to nearest), 128 columns of one row per thread.
constexpr int kPromoteKB = 2;

template <int BN, int STAGES, bool PROMOTE>
__global__ void __launch_bounds__(tc_threads(PROMOTE), 1)
tc_gemm_kernel(const __grid_constant__ TcMaps maps, TcArgs args) {
  constexpr int EPI = epi_warps(PROMOTE);
  constexpr int NBUF = PROMOTE ? 1 : 2;
  static_assert(!PROMOTE || BN == 256, "promoted accumulation: two warps x 128 columns");
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const uint32_t base = smem_u32(smem_raw);
  const uint32_t pad = (1024u - (base & 1023u)) & 1023u;
  auto& S = *reinterpret_cast<TcSmem<BN, STAGES, EPI, NBUF>*>(smem_raw + pad);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tiles_m = (args.M + BM - 1) / BM;
  const int tiles_n = (args.N + BN - 1) / BN;
  const int nk_total = args.nk1 + args.nk2;
  const int nunits = tiles_m * tiles_n * args.splits;
  const int np = args.npairs;
  constexpr uint32_t kStageBytes = (BM + BN) * BK * 2;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&S.full[s], 1);
      mbar_init(&S.empty[s], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&S.acc_full[i], 1);
      mbar_init(&S.acc_empty[i], EPI);
    }
    mbar_init(&S.drain, 1);
    S.abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {   // two accumulators of BN fp32 columns x 128 lanes
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&S.tmem_base)),
                 "r"((uint32_t)(2 * BN)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = S.tmem_base;

  auto unit_k = [&](int u, int& kb0, int& nkb) {
    const int sp = u / (tiles_m * tiles_n);
    kb0 = sp * args.kblocks_per_split;
    nkb = max(0, min(nk_total - kb0, args.kblocks_per_split));
  };

  if (warp == 0) {
    if (lane == 0 && !args.no_loads) {
      // ---------------- producer
      uint32_t g = 0, issued = 0;
      for (int u = blockIdx.x; u < nunits && !*(volatile int*)&S.abort_flag; u += gridDim.x) {
        const int m0 = (u % tiles_m) * BM;
        const int n0 = ((u / tiles_m) % tiles_n) * BN;
        int kb0, nkb;
        unit_k(u, kb0, nkb);
        const int steps = nkb * np;
        for (int kb = 0; kb < steps; ++kb, ++g) {
          const int s = g % STAGES;
          const uint32_t round = g / STAGES;
          if (round > 0 &&
              !mbar_wait_or_abort(&S.empty[s], (round - 1) & 1, 1, &S.abort_flag, args.wait_limit)) {
            S.abort_flag = 1;
            break;
          }
          if (*(volatile int*)&S.abort_flag) break;
          mbar_expect_tx(&S.full[s], kStageBytes);
          const int p = kb % np;
          const int kbg = kb0 + kb / np;
          if (kbg < args.nk1) {
            const int kx = kbg * BK;
            tma_load_2d(&maps.a[args.pa[p]], &S.full[s], S.a[s], kx, m0);
            tma_load_2d(&maps.b[args.pb[p]], &S.full[s], S.b[s], kx, n0);
          } else {   // second segment: K block = (w1, chunk of b')
            const int j = kbg - args.nk1;
            const int w1 = j / args.nbc2, bx = (j % args.nbc2) * BK;
            tma_load_4d(&maps.a2[args.pa[p]], &S.full[s], S.a[s], bx, 0, w1, m0 / args.n12);
            tma_load_3d(&maps.b2[args.pb[p]], &S.full[s], S.b[s], bx, w1, n0);
          }
          issued = g + 1;
        }
      }
      // on abort: wait (bounded) for the copies still in flight before leaving
      if (*(volatile int*)&S.abort_flag) {
        for (uint32_t j = issued > (uint32_t)STAGES ? issued - STAGES : 0; j < issued; ++j)
          mbar_wait(&S.full[j % STAGES], (j / STAGES) & 1, 2, args.wait_limit);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer
      constexpr uint32_t idesc = idesc_bf16(BM, BN);
      uint32_t g = 0, ch = 0;                        // ring steps, accumulator chunks
      bool issued_any = false, ok = true;
      for (int u = blockIdx.x; ok && u < nunits && !*(volatile int*)&S.abort_flag;
           u += gridDim.x) {
        int kb0, nkb;
        unit_k(u, kb0, nkb);
        const int steps = nkb * np;
        const int cs = PROMOTE ? kPromoteKB * np : steps;   // steps per accumulator chunk
        for (int st0 = 0; st0 < steps; st0 += cs, ++ch) {
          const uint32_t buf = ch & 1, use = ch >> 1;
          if (use > 0 &&
              !mbar_wait_or_abort(&S.acc_empty[buf], (use - 1) & 1, 5, &S.abort_flag, args.wait_limit)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t d = tmem + buf * BN;
          const int st1 = min(steps, st0 + cs);
          for (int kb = st0; kb < st1; ++kb, ++g) {
            const int s = g % STAGES;
            if (!mbar_wait_or_abort(&S.full[s], (g / STAGES) & 1, 3, &S.abort_flag, args.wait_limit)) {
              ok = false;
              break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint64_t da = smem_desc(S.a[s]);
            const uint64_t db = smem_desc(S.b[s]);
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk)
              mma_bf16(d, da + (uint64_t)(kk * 2), db + (uint64_t)(kk * 2), idesc,
                       (kb > st0 || kk > 0) ? 1u : 0u);
            issued_any = true;
            mma_commit(&S.empty[s]);   // frees the stage once these MMAs have read it
          }
          if (!ok) break;
          mma_commit(&S.acc_full[buf]);
        }
      }
      if (!ok) S.abort_flag = 1;
      if (*(volatile int*)&S.abort_flag && issued_any) {
        mma_commit(&S.drain);      // wait (bounded) for the MMAs still in flight
        mbar_wait(&S.drain, 0, 6, args.wait_limit);
      }
    }
  } else {
    // ---------------- epilogue warps
    const int q = warp & 3;                          // TMEM lane quarter of this warp
    const int ew = warp - 2;                         // epilogue warp index
    const int colbase = PROMOTE ? (ew >> 2) * 128 : 0;   // columns of this warp (promoted)
    unsigned char* wbuf = S.cbuf[ew][0];             // NBUF x 4 KB, 1024-byte aligned
    const bool bf16_out = args.out_kind == OUT_BF16;
    uint32_t ch = 0, chunk = 0;
    bool ok = true;
    // wait for accumulator chunk `ch` and return its TMEM base
    auto acquire = [&](uint32_t& tl) -> bool {
      const uint32_t buf = ch & 1, use = ch >> 1;
      if (!mbar_wait_or_abort(&S.acc_full[buf], use & 1, 4, &S.abort_flag, args.wait_limit)) return false;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      tl = tmem + buf * BN + (uint32_t)colbase + ((uint32_t)(q * 32) << 16);
      return true;
    };
    auto release = [&]() {
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&S.acc_empty[ch & 1]);
      ++ch;
    };
    // stage one row segment of 32 FP32 values (this lane's row) and store the 32-row slab
    auto store32 = [&](const float (&v)[32], int n0c, int row0) {
      unsigned char* sb = wbuf + (chunk % NBUF) * 4096;
      if (lane == 0) {                    // the store issued from sb NBUF chunks ago
        if (NBUF == 1) bulk_wait_read0();
        else bulk_wait_read1();
      }
      __syncwarp();
      const uint32_t rowa = smem_u32(sb) + lane * 128;
#pragma unroll
      for (int j = 0; j < 8; ++j)
        st_shared_v4(rowa + ((j ^ (lane & 7)) << 4), __float_as_uint(v[4 * j]),
                     __float_as_uint(v[4 * j + 1]), __float_as_uint(v[4 * j + 2]),
                     __float_as_uint(v[4 * j + 3]));
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      // every chunk that wrote a staging buffer commits exactly one bulk group, which is
      // what the wait_group.read accounting above relies on
      if (lane == 0) {
        if (args.out_kind == OUT_F32_ATOMIC) tma_reduce_add_2d(&maps.c, sb, n0c, row0);
        else tma_store_2d(&maps.c, sb, n0c, row0);
        bulk_commit();
      }
      ++chunk;
    };
    // plain stores of one 32 x 32 block through a 4 KB transpose buffer: row r, column c
    // lives at r * 32 + (c ^ r), so that both the row writes and the column reads below
    // touch 32 different banks
    auto plain32 = [&](const float (&v)[32], int n0c, int row0, void* Cb) {
      float* stage = reinterpret_cast<float*>(wbuf);     // (used only without TMA stores)
#pragma unroll
      for (int i = 0; i < 32; ++i) stage[lane * 32 + (i ^ lane)] = v[i];
      __syncwarp();
      const int col = n0c + lane;
      const int nrow = min(32, args.M - row0);
      if (col < args.N) {
        if (args.out_kind == OUT_BF16) {
          __nv_bfloat16* cp =
              reinterpret_cast<__nv_bfloat16*>(Cb) + (long long)row0 * args.ldc + col;
          for (int r = 0; r < nrow; ++r)
            cp[(long long)r * args.ldc] = __float2bfloat16_rn(stage[r * 32 + (lane ^ r)]);
        } else if (args.out_kind == OUT_F32_ATOMIC) {
          float* cp = reinterpret_cast<float*>(Cb) + (long long)row0 * args.ldc + col;
          for (int r = 0; r < nrow; ++r)
            atomicAdd(cp + (long long)r * args.ldc, stage[r * 32 + (lane ^ r)]);
        } else {
          float* cp = reinterpret_cast<float*>(Cb) + (long long)row0 * args.ldc + col;
          for (int r = 0; r < nrow; ++r) cp[(long long)r * args.ldc] = stage[r * 32 + (lane ^ r)];
        }
      }
      __syncwarp();
    };
    for (int u = blockIdx.x; ok && u < nunits; u += gridDim.x) {
      const int m0 = (u % tiles_m) * BM;
      const int n0 = ((u / tiles_m) % tiles_n) * BN;
      const int row0 = m0 + q * 32;
      const bool rows_here = row0 < args.M;
      if constexpr (PROMOTE) {
        int kb0, nkb;
        unit_k(u, kb0, nkb);
        const int steps = nkb * np, cs = kPromoteKB * np;
        float acc[128];
#pragma unroll
        for (int i = 0; i < 128; ++i) acc[i] = 0.f;
        for (int st0 = 0; st0 < steps; st0 += cs) {
          uint32_t tl;
          if (!acquire(tl)) { ok = false; break; }
#pragma unroll
          for (int c0 = 0; c0 < 128; c0 += 32) {
            float v[32];
            tmem_ld32(tl + (uint32_t)c0, v);
#pragma unroll
            for (int i = 0; i < 32; ++i) acc[c0 + i] += v[i];
          }
          release();
        }
        if (!ok) break;
#pragma unroll
        for (int c0 = 0; c0 < 128; c0 += 32) {
          const int col = n0 + colbase + c0;
          if (col < args.N && rows_here) {
            float v[32];
#pragma unroll
            for (int i = 0; i < 32; ++i) v[i] = acc[c0 + i];
            if (args.tma_store) store32(v, col, row0);
            else plain32(v, col, row0, args.C);
          }
        }
      } else {
        uint32_t tl;
        if (!acquire(tl)) { ok = false; break; }
        if (args.tma_store && rows_here) {
          // Each lane owns one row of the 32-row slab: it writes its 128-byte row segment
          // into a 128B-swizzled staging buffer (16-byte chunk j of row r lands at chunk
          // j ^ (r % 8)), then lane 0 issues one TMA store (or reduce-add) of the 32-row
          // box; the box is clipped at the matrix edges by the tensor map.
          const int cw = bf16_out ? 64 : 32;
#pragma unroll 1
          for (int c0 = 0; c0 < BN; c0 += cw) {
            if (n0 + c0 >= args.N) break;
            if (bf16_out) {
              unsigned char* sb = wbuf + (chunk & 1) * 4096;
              if (lane == 0) bulk_wait_read1();
              __syncwarp();
              const uint32_t rowa = smem_u32(sb) + lane * 128;
              float v0[32], v1[32];
              tmem_ld32(tl + (uint32_t)c0, v0);
              tmem_ld32(tl + (uint32_t)(c0 + 32), v1);
#pragma unroll
              for (int j = 0; j < 8; ++j) {
                const float* v = j < 4 ? v0 + 8 * j : v1 + 8 * (j - 4);
                st_shared_v4(rowa + ((j ^ (lane & 7)) << 4), pack_bf16(v[0], v[1]),
                             pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]), pack_bf16(v[6], v[7]));
              }
              asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
              __syncwarp();
              if (lane == 0) {
                tma_store_2d(&maps.c, sb, n0 + c0, row0);
                bulk_commit();
              }
              ++chunk;
            } else {
              float v[32];
              tmem_ld32(tl + (uint32_t)c0, v);
              store32(v, n0 + c0, row0);
            }
          }
        } else if (!args.tma_store) {
          void* Cb = args.C;
          if (args.split_ld > 0)
            Cb = reinterpret_cast<float*>(args.C) + (long long)(u / (tiles_m * tiles_n)) * args.split_ld;
#pragma unroll 1
          for (int c0 = 0; c0 < BN; c0 += 32) {
            if (n0 + c0 >= args.N) break;
            float v[32];
            tmem_ld32(tl + (uint32_t)c0, v);
            plain32(v, n0 + c0, row0, Cb);
          }
        }
        release();
      }
    }
    if (!ok) S.abort_flag = 1;
    if (args.tma_store && lane == 0) bulk_wait_all();   // stores complete before exit
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"((uint32_t)(2 * BN)));
  }
}

// ------------------------------------------------------------------ host side
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  if (!fn) throw CudaError("cuTensorMapEncodeTiled unavailable");
  return fn;
}

// 2D K-major BF16 operand: rows x K (row stride ld elements), box BK x box_rows, 128B swizzle.
CUtensorMap make_map(const __nv_bfloat16* ptr, int rows, int K, long long ld, int box_rows) {
  A2_REQUIRE((reinterpret_cast<uintptr_t>(ptr) & 15) == 0, "TMA base must be 16-byte aligned");
  A2_REQUIRE((ld * 2) % 16 == 0, "TMA row stride must be a multiple of 16 bytes");
  CUtensorMap m;
  cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
  cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)ptr, dims, strides,
                           box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) throw CudaError("cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
  return m;
}

// Tiled BF16 map of rank 3 or 4 (dims innermost first, strides in bytes for dims 1..),
// 128B swizzle, zero fill outside the extents.
CUtensorMap make_map_nd(const __nv_bfloat16* ptr, int rank, const cuuint64_t* dims,
                        const cuuint64_t* strides, const cuuint32_t* box) {
  A2_REQUIRE((reinterpret_cast<uintptr_t>(ptr) & 15) == 0, "TMA base must be 16-byte aligned");
  for (int i = 0; i < rank - 1; ++i)
    A2_REQUIRE(strides[i] % 16 == 0, "TMA strides must be multiples of 16 bytes");
  CUtensorMap m;
  cuuint32_t estr[4] = {1, 1, 1, 1};
  CUresult r = encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, rank, (void*)ptr, dims, strides,
                           box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) throw CudaError("cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
  return m;
}

// Returns the number of K splits launched.  split_ld > 0: every split stores its own FP32
// tile at C + sp * split_ld (plain stores), with at most `splitk`-derived K blocks each.
template <int BN, int STAGES, bool PROMOTE>
int launch(const __nv_bfloat16* const* A, long long lda, const __nv_bfloat16* const* B,
           long long ldb, int M, int N, int K, int npairs, const int* pa, const int* pb,
           const TcSeg2* seg, void* C, long long ldc, int out_kind, int splitk,
           cudaStream_t s, long long split_ld = 0) {
  A2_REQUIRE(npairs >= 1 && npairs <= kMaxPairs, "tc GEMM: 1..8 operand pairs");
  TcMaps maps;
  int na = 0, nb = 0;
  for (int p = 0; p < npairs; ++p) {
    A2_REQUIRE(pa[p] >= 0 && pa[p] < kMaxPlanes && pb[p] >= 0 && pb[p] < kMaxPlanes,
               "tc GEMM: plane index out of range");
    na = std::max(na, pa[p] + 1);
    nb = std::max(nb, pb[p] + 1);
  }
  for (int i = 0; i < kMaxPlanes; ++i) {
    maps.a[i] = i < na || i == 0 ? make_map(A[i], M, K, lda, BM) : maps.a[0];
    maps.b[i] = i < nb || i == 0 ? make_map(B[i], N, K, ldb, BN) : maps.b[0];
  }
  int nk2 = 0, nbc2 = 1, n12 = 1;
  if (seg) {
    const long long Dr = seg->Dr, R1 = seg->R1;
    n12 = seg->n12;
    A2_REQUIRE(n12 >= 1 && BM % n12 == 0 && (long long)M == (long long)seg->Dl * n12,
               "tc GEMM segment: rows must be (a, s12) with s12 dividing 128");
    A2_REQUIRE(Dr % 8 == 0 && seg->Nb == N, "tc GEMM segment: Dr % 8 == 0, N == Dr");
    nbc2 = (int)((Dr + BK - 1) / BK);
    nk2 = (int)(R1 * nbc2);
    for (int i = 0; i < 3; ++i) {
      const cuuint64_t ad[4] = {(cuuint64_t)Dr, (cuuint64_t)n12, (cuuint64_t)R1,
                                (cuuint64_t)seg->Dl};
      const cuuint64_t as[3] = {(cuuint64_t)(Dr * 2), (cuuint64_t)(n12 * Dr * 2),
                                (cuuint64_t)(R1 * n12 * Dr * 2)};
      const cuuint32_t ab[4] = {(cuuint32_t)BK, (cuuint32_t)n12, 1u, (cuuint32_t)(BM / n12)};
      maps.a2[i] = make_map_nd(seg->A[i < na ? i : 0], 4, ad, as, ab);
      const cuuint64_t bd[3] = {(cuuint64_t)Dr, (cuuint64_t)R1, (cuuint64_t)N};
      const cuuint64_t bs[2] = {(cuuint64_t)(Dr * 2), (cuuint64_t)(R1 * Dr * 2)};
      const cuuint32_t bb[3] = {(cuuint32_t)BK, 1u, (cuuint32_t)BN};
      maps.b2[i] = make_map_nd(seg->B[i < nb ? i : 0], 3, bd, bs, bb);
    }
  } else {
    for (int i = 0; i < 3; ++i) {
      maps.a2[i] = maps.a[i];
      maps.b2[i] = maps.b[i];
    }
  }
  constexpr int EPI = epi_warps(PROMOTE);
  const size_t smem = sizeof(TcSmem<BN, STAGES, EPI, PROMOTE ? 1 : 2>) + 1024;
  static std::once_flag once;
  std::call_once(once, [smem] {
    A2_CUDA(cudaFuncSetAttribute(tc_gemm_kernel<BN, STAGES, PROMOTE>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  });
  static int num_sms = 0;
  static std::once_flag sms_once;
  std::call_once(sms_once, [] {
    int dev = 0;
    A2_CUDA(cudaGetDevice(&dev));
    A2_CUDA(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev));
  });
  const int nk1 = (K + BK - 1) / BK;
  const int nk_total = nk1 + nk2;
  splitk = std::max(1, std::min(splitk, nk_total));
  TcArgs args;
  args.M = M; args.N = N; args.K = K;
  args.nk1 = nk1; args.nk2 = nk2; args.nbc2 = nbc2; args.n12 = n12;
  args.kblocks_per_split = (nk_total + splitk - 1) / splitk;
  splitk = (nk_total + args.kblocks_per_split - 1) / args.kblocks_per_split;
  args.C = C; args.ldc = ldc; args.out_kind = out_kind;
  args.npairs = npairs;
  for (int p = 0; p < kMaxPairs; ++p) {
    args.pa[p] = p < npairs ? pa[p] : 0;
    args.pb[p] = p < npairs ? pb[p] : 0;
  }
  args.splits = splitk;
  args.split_ld = split_ld;
  args.wait_limit = kWaitLimit;
  args.no_loads = 0;
  A2_REQUIRE(split_ld == 0 || (out_kind == OUT_F32 && !PROMOTE), "split tiles: FP32 stores");
  // TMA store epilogue when C's base and row stride allow it
  {
    const size_t es = out_kind == OUT_BF16 ? 2 : 4;
    args.tma_store = ((reinterpret_cast<uintptr_t>(C) & 15) == 0 && (ldc * es) % 16 == 0 &&
                      ldc >= N && split_ld == 0) ? 1 : 0;
    if (args.tma_store) {
      const cuuint64_t cd[2] = {(cuuint64_t)N, (cuuint64_t)M};
      const cuuint64_t cs[1] = {(cuuint64_t)(ldc * es)};
      const cuuint32_t cb[2] = {(cuuint32_t)(out_kind == OUT_BF16 ? 64 : 32), 32u};
      const cuuint32_t ce[2] = {1, 1};
      CUresult r = encode_fn()(&maps.c,
                               out_kind == OUT_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                    : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                               2, C, cd, cs, cb, ce, CU_TENSOR_MAP_INTERLEAVE_NONE,
                               CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS) args.tma_store = 0;
    }
  }
  const long long units = (long long)cdiv(M, BM) * cdiv(N, BN) * splitk;
  A2_REQUIRE(units < (1LL << 31), "tcgen05 GEMM too large");
  const int grid = (int)std::min<long long>(units, std::max(1, num_sms));
  tc_gemm_kernel<BN, STAGES, PROMOTE><<<grid, tc_threads(PROMOTE), smem, s>>>(maps, args);
  A2_CHECK_LAUNCH();
  return splitk;
}

// ------------------------------------------------------------------ Ozaki GEMM, register sums
// FP64-class product of two operands given as kOzSlices BF16 slice planes each (the
// slicing of the FP64 emulation below).  Work unit = (128 x 128 output tile, K split).
// For every level l = 2 .. kOzSlices + 1 the l - 1 slice pairs of that level are
// accumulated over chunks of at most 16 / (l - 1) K blocks into a fresh TMEM buffer: a
// chunk holds at most 1024 products per output element, each an integer multiple of the
// level's unit below 2^14 units, so its FP32 sum is exact.  The epilogue adds every chunk
// into a double-float register accumulator (hi + lo, Knuth's error-free two-sum), so no
// per-level tile reaches memory.  Warp 0 lane 0: TMA producer; warp 1 lane 0: MMA issuer;
// warps 2..9: epilogue (two per TMEM lane quarter, 64 columns each).  Every wait is
// bounded as in tc_gemm_kernel.
constexpr int kOzBN = 128;
constexpr int kOzStages = 5;
constexpr int kOzEpi = 8;
constexpr int kOzThreads = 64 + 32 * kOzEpi;
constexpr int kOzMaxLevel = 9;                  // slice pairs (i, j) with i + j <= 9

struct OzSmem {
  alignas(1024) __nv_bfloat16 a[kOzStages][BM * BK];
  alignas(1024) __nv_bfloat16 b[kOzStages][kOzBN * BK];
  alignas(1024) float stage[kOzEpi][2][32 * 32];   // epilogue transpose buffers (hi, lo)
  alignas(8) uint64_t full[kOzStages];
  alignas(8) uint64_t empty[kOzStages];
  alignas(8) uint64_t acc_full[2];
  alignas(8) uint64_t acc_empty[2];
  alignas(8) uint64_t drain;
  uint32_t tmem_base;
  int abort_flag;
};
static_assert(sizeof(OzSmem) + 1024 <= 227 * 1024, "Ozaki ring exceeds shared memory");

enum OzOut { OZ_F64 = 0, OZ_PAIR = 1, OZ_SPLIT = 2 };

struct OzArgs {
  int M, N, nk;              // rows, columns, K blocks of BK
  int kblocks_per_split, splits;
  int n_fast;                // 1: consecutive units walk the N tiles of one row of tiles
  int out_mode;              // OZ_F64: C[m*ldc + n] = hi + lo (FP64)
                             // OZ_PAIR: FP32 hi at C[m*ldc + n], lo at + df_plane
                             // OZ_SPLIT: FP32 tiles of split sp, hi at C + 2sp*MN and lo at
                             //           C + (2sp+1)*MN, row stride N
  void* C;
  long long ldc, df_plane, MN;
};

__device__ __forceinline__ int oz_chunk_blocks(int np) { return max(1, 16 / np); }

// 10 warps: three of them share one SM sub-partition's 16K registers, hence at most 168
// registers per thread.
__global__ void __launch_bounds__(kOzThreads, 1)
tc_oz_kernel(const __grid_constant__ TcMaps maps, OzArgs args) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const uint32_t base = smem_u32(smem_raw);
  const uint32_t pad = (1024u - (base & 1023u)) & 1023u;
  auto& S = *reinterpret_cast<OzSmem*>(smem_raw + pad);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tiles_m = (args.M + BM - 1) / BM;
  const int tiles_n = (args.N + kOzBN - 1) / kOzBN;
  const int nunits = tiles_m * tiles_n * args.splits;
  constexpr uint32_t kStageBytes = (BM + kOzBN) * BK * 2;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kOzStages; ++s) {
      mbar_init(&S.full[s], 1);
      mbar_init(&S.empty[s], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&S.acc_full[i], 1);
      mbar_init(&S.acc_empty[i], kOzEpi);
    }
    mbar_init(&S.drain, 1);
    S.abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {   // two accumulators of 128 fp32 columns x 128 lanes
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&S.tmem_base)),
                 "r"((uint32_t)(2 * kOzBN)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = S.tmem_base;

  auto unit = [&](int u, int& m0, int& n0, int& kb0, int& nkb) {
    const int t = u % (tiles_m * tiles_n), sp = u / (tiles_m * tiles_n);
    if (args.n_fast) {
      n0 = (t % tiles_n) * kOzBN;
      m0 = (t / tiles_n) * BM;
    } else {
      m0 = (t % tiles_m) * BM;
      n0 = (t / tiles_m) * kOzBN;
    }
    kb0 = sp * args.kblocks_per_split;
    nkb = max(0, min(args.nk - kb0, args.kblocks_per_split));
  };

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- producer: level, chunk, K block, slice pair
      uint32_t g = 0, issued = 0;
      bool stop = false;
      for (int u = blockIdx.x; !stop && u < nunits && !*(volatile int*)&S.abort_flag;
           u += gridDim.x) {
        int m0, n0, kb0, nkb;
        unit(u, m0, n0, kb0, nkb);
        for (int l = 2; !stop && l <= kOzMaxLevel; ++l) {
          const int np = l - 1, kbl = oz_chunk_blocks(np);
          for (int c0 = 0; !stop && c0 < nkb; c0 += kbl) {
            const int c1 = min(nkb, c0 + kbl);
            for (int kb = c0; !stop && kb < c1; ++kb) {
              for (int p = 0; p < np; ++p, ++g) {
                const int s = g % kOzStages;
                const uint32_t round = g / kOzStages;
                if ((round > 0 &&
                     !mbar_wait_or_abort(&S.empty[s], (round - 1) & 1, 11, &S.abort_flag)) ||
                    *(volatile int*)&S.abort_flag) {
                  S.abort_flag = 1;
                  stop = true;
                  break;
                }
                mbar_expect_tx(&S.full[s], kStageBytes);
                const int kx = (kb0 + kb) * BK;
                tma_load_2d(&maps.a[p], &S.full[s], S.a[s], kx, m0);
                tma_load_2d(&maps.b[np - 1 - p], &S.full[s], S.b[s], kx, n0);
                issued = g + 1;
              }
            }
          }
        }
      }
      if (*(volatile int*)&S.abort_flag) {   // wait (bounded) for the copies in flight
        for (uint32_t j = issued > (uint32_t)kOzStages ? issued - kOzStages : 0; j < issued; ++j)
          mbar_wait(&S.full[j % kOzStages], (j / kOzStages) & 1, 12);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer: one TMEM buffer per (level, chunk)
      constexpr uint32_t idesc = idesc_bf16(BM, kOzBN);
      uint32_t g = 0, ch = 0;
      bool issued_any = false, ok = true;
      for (int u = blockIdx.x; ok && u < nunits && !*(volatile int*)&S.abort_flag;
           u += gridDim.x) {
        int m0, n0, kb0, nkb;
        unit(u, m0, n0, kb0, nkb);
        for (int l = 2; ok && l <= kOzMaxLevel; ++l) {
          const int np = l - 1, kbl = oz_chunk_blocks(np);
          for (int c0 = 0; ok && c0 < nkb; c0 += kbl, ++ch) {
            const int c1 = min(nkb, c0 + kbl);
            const uint32_t buf = ch & 1, use = ch >> 1;
            if (use > 0 &&
                !mbar_wait_or_abort(&S.acc_empty[buf], (use - 1) & 1, 13, &S.abort_flag)) {
              ok = false;
              break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t d = tmem + buf * kOzBN;
            bool first = true;
            for (int kb = c0; ok && kb < c1; ++kb) {
              for (int p = 0; p < np; ++p, ++g) {
                const int s = g % kOzStages;
                if (!mbar_wait_or_abort(&S.full[s], (g / kOzStages) & 1, 14, &S.abort_flag)) {
                  ok = false;
                  break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint64_t da = smem_desc(S.a[s]);
                const uint64_t db = smem_desc(S.b[s]);
#pragma unroll
                for (int kk = 0; kk < BK / 16; ++kk)
                  mma_bf16(d, da + (uint64_t)(kk * 2), db + (uint64_t)(kk * 2), idesc,
                           (first && kk == 0) ? 0u : 1u);
                first = false;
                issued_any = true;
                mma_commit(&S.empty[s]);
              }
            }
            if (!ok) break;
            mma_commit(&S.acc_full[buf]);
          }
        }
      }
      if (!ok) S.abort_flag = 1;
      if (*(volatile int*)&S.abort_flag && issued_any) {
        mma_commit(&S.drain);
        mbar_wait(&S.drain, 0, 15);
      }
    }
  } else {
    // ---------------- epilogue: double-float sums of the chunks, then the output
    const int q = warp & 3;                 // TMEM lane quarter of this warp
    const int ew = warp - 2;
    const int colbase = (ew >> 2) * 64;     // this warp's 64 columns of the tile
    float* sh = S.stage[ew][0];
    float* sl = S.stage[ew][1];
    uint32_t ch = 0;
    bool ok = true;
    for (int u = blockIdx.x; ok && u < nunits; u += gridDim.x) {
      int m0, n0, kb0, nkb;
      unit(u, m0, n0, kb0, nkb);
      float hi[64], lo[64];
#pragma unroll
      for (int i = 0; i < 64; ++i) hi[i] = lo[i] = 0.f;
      for (int l = 2; ok && l <= kOzMaxLevel; ++l) {
        const int kbl = oz_chunk_blocks(l - 1);
        for (int c0 = 0; c0 < nkb; c0 += kbl, ++ch) {
          const uint32_t buf = ch & 1, use = ch >> 1;
          if (!mbar_wait_or_abort(&S.acc_full[buf], use & 1, 16, &S.abort_flag)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t tl = tmem + buf * kOzBN + (uint32_t)colbase + ((uint32_t)(q * 32) << 16);
#pragma unroll
          for (int c = 0; c < 64; c += 8) {
            float v[8];
            tmem_ld8(tl + (uint32_t)c, v);
#pragma unroll
            for (int i = 0; i < 8; ++i) {   // (hi, lo) += v exactly up to lo's rounding
              const float sum = __fadd_rn(hi[c + i], v[i]);
              const float bp = __fsub_rn(sum, hi[c + i]);
              const float err =
                  __fadd_rn(__fsub_rn(hi[c + i], __fsub_rn(sum, bp)), __fsub_rn(v[i], bp));
              hi[c + i] = sum;
              lo[c + i] = __fadd_rn(lo[c + i], err);
            }
          }
          asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
          __syncwarp();
          if (lane == 0) mbar_arrive(&S.acc_empty[buf]);
        }
      }
      if (!ok) break;
      // output: 32 x 32 blocks through the transpose buffers (lane = row on the way in,
      // lane = column on the way out), so that every store instruction is coalesced
      const int row0 = m0 + q * 32;
#pragma unroll
      for (int c = 0; c < 64; c += 32) {
        const int col0 = n0 + colbase + c;
        if (col0 >= args.N || row0 >= args.M) continue;
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          sh[lane * 32 + (i ^ lane)] = hi[c + i];
          sl[lane * 32 + (i ^ lane)] = lo[c + i];
        }
        __syncwarp();
        const int col = col0 + lane;
        const int nrow = min(32, args.M - row0);
        if (col < args.N) {
          if (args.out_mode == OZ_F64) {
            double* cp = reinterpret_cast<double*>(args.C) + (long long)row0 * args.ldc + col;
#pragma unroll 4
            for (int r = 0; r < nrow; ++r)
              cp[(long long)r * args.ldc] =
                  (double)sh[r * 32 + (lane ^ r)] + (double)sl[r * 32 + (lane ^ r)];
          } else if (args.out_mode == OZ_PAIR) {
            float* cp = reinterpret_cast<float*>(args.C) + (long long)row0 * args.ldc + col;
#pragma unroll 4
            for (int r = 0; r < nrow; ++r) {
              const float h = sh[r * 32 + (lane ^ r)], e = sl[r * 32 + (lane ^ r)];
              const float sum = __fadd_rn(h, e);   // renormalised pair
              cp[(long long)r * args.ldc] = sum;
              cp[(long long)r * args.ldc + args.df_plane] = __fsub_rn(e, __fsub_rn(sum, h));
            }
          } else {
            const int sp = u / (tiles_m * tiles_n);
            float* cp = reinterpret_cast<float*>(args.C) + 2LL * sp * args.MN +
                        (long long)row0 * args.N + col;
#pragma unroll 4
            for (int r = 0; r < nrow; ++r) {
              cp[(long long)r * args.N] = sh[r * 32 + (lane ^ r)];
              cp[(long long)r * args.N + args.MN] = sl[r * 32 + (lane ^ r)];
            }
          }
        }
        __syncwarp();
      }
    }
    if (!ok) S.abort_flag = 1;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"((uint32_t)(2 * kOzBN)));
  }
}

// Launches tc_oz_kernel over planes A[0..7] (M x K, row stride lda) and B[0..7] (N x K).
void launch_oz(const __nv_bfloat16* const* A, long long lda, const __nv_bfloat16* const* B,
               long long ldb, int M, int N, int K, int splits, int out_mode, void* C,
               long long ldc, long long df_plane, cudaStream_t s) {
  TcMaps maps;
  for (int i = 0; i < kMaxPlanes; ++i) {
    maps.a[i] = make_map(A[i], M, K, lda, BM);
    maps.b[i] = make_map(B[i], N, K, ldb, kOzBN);
  }
  for (int i = 0; i < 3; ++i) {
    maps.a2[i] = maps.a[i];
    maps.b2[i] = maps.b[i];
  }
  maps.c = maps.a[0];
  const size_t smem = sizeof(OzSmem) + 1024;
  static std::once_flag once;
  std::call_once(once, [smem] {
    A2_CUDA(cudaFuncSetAttribute(tc_oz_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
  });
  static int num_sms = 0;
  static std::once_flag sms_once;
  std::call_once(sms_once, [] {
    int dev = 0;
    A2_CUDA(cudaGetDevice(&dev));
    A2_CUDA(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev));
  });
  OzArgs args;
  args.M = M; args.N = N;
  args.nk = (K + BK - 1) / BK;
  splits = std::max(1, std::min(splits, args.nk));
  args.kblocks_per_split = (args.nk + splits - 1) / splits;
  args.splits = (args.nk + args.kblocks_per_split - 1) / args.kblocks_per_split;
  A2_REQUIRE(args.splits == 1 || out_mode == OZ_SPLIT, "Ozaki GEMM: K splits need split tiles");
  args.n_fast = cdiv(N, kOzBN) <= 64 ? 1 : 0;
  args.out_mode = out_mode;
  args.C = C; args.ldc = ldc; args.df_plane = df_plane;
  args.MN = (long long)M * N;
  const long long units = (long long)cdiv(M, BM) * cdiv(N, kOzBN) * args.splits;
  A2_REQUIRE(units < (1LL << 31), "Ozaki GEMM too large");
  const int grid = (int)std::min<long long>(units, std::max(1, num_sms));
  tc_oz_kernel<<<grid, kOzThreads, smem, s>>>(maps, args);
  A2_CHECK_LAUNCH();
}

}  // namespace tc

bool tc_available() { return true; }

int tc_error_flag(bool reset) {
  int v = 0;
  A2_CUDA(cudaMemcpyFromSymbol(&v, tc::g_tc_error, sizeof(int)));
  if (reset && v) {
    int z = 0;
    A2_CUDA(cudaMemcpyToSymbol(tc::g_tc_error, &z, sizeof(int)));
  }
  return v;
}

int tc_selftest_timeout(cudaStream_t s) {
  // One 128 x 128 x 128 unit of the BF16 GEMM kernel whose producer issues no copies: the
  // MMA role's first wait (stage 0 full) can never complete, gives up after 2^14
  // iterations, raises the error word and the abort flag; the epilogue roles see the flag
  // and leave; no copy or MMA is ever in flight and TMEM is freed as on any abort.
  constexpr int n = 128;
  DevBuf a, b, c;
  a.ensure(sizeof(__nv_bfloat16) * n * n, s);
  b.ensure(sizeof(__nv_bfloat16) * n * n, s);
  c.ensure(sizeof(float) * n * n, s);
  fill_zero(a.p, sizeof(__nv_bfloat16) * n * n, s);
  fill_zero(b.p, sizeof(__nv_bfloat16) * n * n, s);
  tc::TcMaps maps;
  for (int i = 0; i < tc::kMaxPlanes; ++i) {
    maps.a[i] = tc::make_map(a.as<__nv_bfloat16>(), n, n, n, tc::BM);
    maps.b[i] = tc::make_map(b.as<__nv_bfloat16>(), n, n, n, 128);
  }
  for (int i = 0; i < 3; ++i) {
    maps.a2[i] = maps.a[i];
    maps.b2[i] = maps.b[i];
  }
  maps.c = maps.a[0];
  tc::TcArgs args{};
  args.M = args.N = args.K = n;
  args.nk1 = n / tc::BK;
  args.nk2 = 0;
  args.nbc2 = args.n12 = 1;
  args.kblocks_per_split = args.nk1;
  args.splits = 1;
  args.C = c.p;
  args.ldc = n;
  args.out_kind = tc::OUT_F32;
  args.npairs = 1;
  args.tma_store = 0;
  args.split_ld = 0;
  args.wait_limit = 1u << 14;
  args.no_loads = 1;
  const size_t smem = sizeof(tc::TcSmem<128, 6, 4, 2>) + 1024;
  A2_CUDA(cudaFuncSetAttribute(tc::tc_gemm_kernel<128, 6, false>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  tc::tc_gemm_kernel<128, 6, false><<<1, tc::tc_threads(false), smem, s>>>(maps, args);
  A2_CHECK_LAUNCH();
  A2_CUDA(cudaStreamSynchronize(s));
  return tc_error_flag(true);
}

void tc_gemm_bf16(const __nv_bfloat16* A, long long lda, const __nv_bfloat16* B, long long ldb,
                  int M, int N, int K, void* C, long long ldc, int out_kind, int splitk,
                  cudaStream_t s) {
  const __nv_bfloat16* Ap[3] = {A, A, A};
  const __nv_bfloat16* Bp[3] = {B, B, B};
  const int p0[1] = {0};
  tc_gemm_bf16_pairs(Ap, lda, Bp, ldb, M, N, K, 1, p0, p0, C, ldc, out_kind, splitk, s);
}

namespace {

// One GEMM configuration: the kernel variant (0: BN = 128 / 6 stages, 1: BN = 256 /
// 4 stages, 2: promoted split products) and the number of K splits.
struct TcConfig {
  int variant = 1, splitk = 1;
};

void run_config(const TcConfig& cfg, const __nv_bfloat16* const* A, long long lda,
                const __nv_bfloat16* const* B, long long ldb, int M, int N, int K, int npairs,
                const int* pa, const int* pb, void* C, long long ldc, int out_kind,
                cudaStream_t s, const TcSeg2* seg) {
  if (cfg.variant == 2)
    tc::launch<256, 4, true>(A, lda, B, ldb, M, N, K, npairs, pa, pb, seg, C, ldc, out_kind,
                             cfg.splitk, s);
  else if (cfg.variant == 0)
    tc::launch<128, 6, false>(A, lda, B, ldb, M, N, K, npairs, pa, pb, seg, C, ldc, out_kind,
                              cfg.splitk, s);
  else
    tc::launch<256, 4, false>(A, lda, B, ldb, M, N, K, npairs, pa, pb, seg, C, ldc, out_kind,
                              cfg.splitk, s);
}

// Autotuner: the first call of a GEMM shape class (tile counts of M and N, K in steps of
// 512, operand pairs, output kind, second segment) times the candidate configurations
// with CUDA events on the caller's stream and keeps the fastest for every later call of
// that class.  Candidates: the kernel
// variants that apply (BN = 128 / 256; the promoted kernel for split products) and, for
// accumulated outputs, the caller's K-split count, half and twice it.  Trials with an
// accumulated output re-zero C first; the winner then runs on a zeroed C.
struct TuneKey {
  int M, N, K, npairs, out_kind, seg_rows;
  bool operator<(const TuneKey& o) const {
    return std::tie(M, N, K, npairs, out_kind, seg_rows) <
           std::tie(o.M, o.N, o.K, o.npairs, o.out_kind, o.seg_rows);
  }
};
std::mutex g_tune_mu;
std::map<TuneKey, TcConfig> g_tune;
bool g_tune_on = true;

}  // namespace

void tc_autotune(bool on) {
  std::lock_guard<std::mutex> g(g_tune_mu);
  g_tune_on = on;
  if (!on) g_tune.clear();
}

void tc_gemm_bf16_pairs(const __nv_bfloat16* const* A, long long lda,
                        const __nv_bfloat16* const* B, long long ldb, int M, int N, int K,
                        int npairs, const int* pa, const int* pb, void* C, long long ldc,
                        int out_kind, int splitk, cudaStream_t s, const TcSeg2* seg) {
  if (M <= 0 || N <= 0) return;
  A2_REQUIRE(K >= 1 && npairs >= 1 && npairs <= 6, "tc GEMM: K >= 1, 1..6 operand pairs");
  if (splitk > 1)
    A2_REQUIRE(out_kind == tc::OUT_F32_ATOMIC, "split-K needs atomic FP32 output");
  const bool promote = npairs > 1 && out_kind != tc::OUT_BF16;  // split products: promoted sums
  TcConfig def;
  def.variant = promote ? 2 : (N <= 128 ? 0 : 1);
  def.splitk = splitk;
  // shapes with the same tile counts (and K within 512) share one decision
  const TuneKey key{(M + 127) / 128, (N + 127) / 128, (K + 511) / 512, npairs, out_kind,
                    seg ? (seg->R1 * seg->Dr + 511) / 512 : 0};
  bool tune = false;
  TcConfig best = def;
  {
    std::lock_guard<std::mutex> g(g_tune_mu);
    if (g_tune_on) {
      auto it = g_tune.find(key);
      if (it != g_tune.end()) best = it->second;
      else tune = true;
    }
  }
  if (!tune) {
    run_config(best, A, lda, B, ldb, M, N, K, npairs, pa, pb, C, ldc, out_kind, s, seg);
    return;
  }
  std::vector<TcConfig> cand;
  std::vector<int> variants = promote ? std::vector<int>{2} : std::vector<int>{0, 1};
  std::vector<int> splits{splitk};
  if (out_kind == tc::OUT_F32_ATOMIC) {
    splits.push_back(splitk * 2);
    if (splitk > 1) splits.push_back(std::max(1, splitk / 2));
  }
  for (int v : variants)
    for (int k : splits) cand.push_back(TcConfig{v, k});
  const size_t cbytes = (size_t)M * ldc * (out_kind == tc::OUT_BF16 ? 2 : 4);
  cudaEvent_t e0, e1;
  A2_CUDA(cudaEventCreate(&e0));
  A2_CUDA(cudaEventCreate(&e1));
  float best_ms = 1e30f;
  for (const TcConfig& cf : cand) {
    if (out_kind == tc::OUT_F32_ATOMIC) fill_zero(C, cbytes, s);
    A2_CUDA(cudaEventRecord(e0, s));
    run_config(cf, A, lda, B, ldb, M, N, K, npairs, pa, pb, C, ldc, out_kind, s, seg);
    A2_CUDA(cudaEventRecord(e1, s));
    A2_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    A2_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    if (ms < best_ms) {
      best_ms = ms;
      best = cf;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  {
    std::lock_guard<std::mutex> g(g_tune_mu);
    g_tune[key] = best;
  }
  if (out_kind == tc::OUT_F32_ATOMIC) fill_zero(C, cbytes, s);
  run_config(best, A, lda, B, ldb, M, N, K, npairs, pa, pb, C, ldc, out_kind, s, seg);
}

// -------------------------------------------------------------- BF16 H_eff chain
namespace {
int s4_splitk(long long M4, int Dr, long long kblocks) {
  const long long tiles = (long long)cdiv(M4, 128) * cdiv(Dr, Dr <= 128 ? 128 : 256);
  int splitk = (int)std::max<long long>(1, 2 * 152 / std::max<long long>(1, tiles));
  return std::min<int>(splitk, std::max<int>(1, (int)(kblocks / 8)));
}
}  // namespace

void tc_heff_bf16(cudaStream_t s, int n1, int n2, int Rl, int R1, int Rr, int Dl, int Dr,
                  const __nv_bfloat16* Lb, long long ldl, const __nv_bfloat16* Rb, long long ldr,
                  const double* x, float* y, const SparseRows<float>& W1,
                  const SparseRows<float>& W2, const HeffFold& F, DevBuf& t1, DevBuf& t2,
                  DevBuf& xa, DevBuf& tf) {
  (void)tf;
  const long long NX = (long long)n1 * n2 * Dr;          // columns of S1
  const long long ldx = pad8(Dl);
  const long long s1 = (long long)Dl * Rl * NX;
  const long long s2 = (long long)Dl * R1 * NX;
  const long long K4 = (long long)Rr * Dr;
  const long long ld3 = pad8(K4);
  const long long s3 = (long long)Dl * n1 * n2 * ld3;
  xa.ensure(sizeof(__nv_bfloat16) * (size_t)NX * ldx, s);
  t1.ensure(sizeof(__nv_bfloat16) * (size_t)std::max(s1, s3), s);
  t2.ensure(sizeof(__nv_bfloat16) * (size_t)s2, s);
  __nv_bfloat16* XT = xa.as<__nv_bfloat16>();
  __nv_bfloat16* T1 = t1.as<__nv_bfloat16>();
  __nv_bfloat16* T2 = t2.as<__nv_bfloat16>();
  __nv_bfloat16* T3 = t1.as<__nv_bfloat16>();
  // x [Dl][(t1 t2 b')] -> XT [(t1 t2 b')][a'] (row stride ldx)
  // (pad columns a' >= Dl are never read: the tensor map's K extent is Dl)
  transpose2d_ld<double, __nv_bfloat16>(x, XT, Dl, (int)NX, ldx, s);
  // S1: T1[(a w)][(t1 t2 b')] = sum_a' L[(a w)][a'] XT[(t1 t2 b')][a']
  {
    const double M = (double)Dl * Rl, N = (double)NX, K = Dl;
    ProfScope ps(PK_TC_S1, s, 2.0 * M * N * K, 2.0 * (M * K + N * K + M * N));
    tc_gemm_bf16(Lb, ldl, XT, ldx, Dl * Rl, (int)NX, Dl, T1, NX, tc::OUT_BF16, 1, s);
  }
  if (F.Lt) {   // folded G of A_k: T2[(a w1)][(s1 t2 b')] = sum_a' Lt[(a w1)][a'] XT
    const double M = (double)Dl * R1, N = (double)NX, K = Dl;
    ProfScope ps(PK_TC_S1, s, 2.0 * M * N * K, 2.0 * (M * K + N * K + M * N));
    tc_gemm_bf16(F.Lt, ldl, XT, ldx, Dl * R1, (int)NX, Dl, T2, NX, tc::OUT_BF16, 1, s);
  }
  {  // S2 (W_rest added to the folded part when A_k is folded)
    ProfScope ps(PK_SPARSE_S2, s, 2.0 * W1.nnz_total * (double)n2 * Dr * Dl,
                 2.0 * (double)(s1 + s2) * (F.Lt ? 1.5 : 1.0));
    SparseGeom gm;
    gm.veclen = n2 * Dr;
    gm.in_sw = NX; gm.in_st = (long long)n2 * Dr;
    gm.out_sw = NX; gm.out_ss = (long long)n2 * Dr;
    gm.B1 = Dl; gm.in_b1 = (long long)Rl * NX; gm.out_b1 = (long long)R1 * NX;
    gm.accumulate = F.Lt ? 1 : 0;
    sparse_rows_apply<__nv_bfloat16, __nv_bfloat16, float>(W1, gm, T1, T2, s);
  }
  {  // S3 -> T3[(a s1 s2)][(w2 b')] with row stride ld3
    ProfScope ps(PK_SPARSE_S3, s, 2.0 * W2.nnz_total * (double)Dr * Dl * n1,
                 2.0 * (double)s2 + 2.0 * (double)Dl * n1 * n2 * Rr * Dr);
    SparseGeom gm;
    gm.veclen = Dr;
    gm.in_sw = NX; gm.in_st = Dr;
    gm.out_sw = Dr; gm.out_ss = ld3;
    gm.B1 = Dl; gm.B2 = n1;
    gm.in_b1 = (long long)R1 * NX; gm.in_b2 = (long long)n2 * Dr;
    gm.out_b1 = (long long)n1 * n2 * ld3; gm.out_b2 = (long long)n2 * ld3;
    sparse_rows_apply<__nv_bfloat16, __nv_bfloat16, float>(W2, gm, T2, T3, s);
  }
  // S4: y[(a s1 s2)][b] = sum_{(w2 b')} T3 HR[b][(w2 b')]   (split K, atomic FP32)
  //     (+ sum_{(w1 b')} T2[a][w1][(s1 s2)][b'] Rt[b][w1][b'] when A_{k+1} is folded)
  const int M4 = Dl * n1 * n2;
  TcSeg2 seg;
  long long kb = (K4 + 63) / 64;
  if (F.Rt) {
    seg.A[0] = seg.A[1] = seg.A[2] = T2;
    seg.B[0] = seg.B[1] = seg.B[2] = F.Rt;
    seg.Dl = Dl; seg.n12 = n1 * n2; seg.R1 = R1; seg.Dr = Dr; seg.Nb = Dr;
    kb += (long long)R1 * ((Dr + 63) / 64);
  }
  {
    const double M = M4, N = Dr, K = (double)K4 + (F.Rt ? (double)R1 * Dr : 0.0);
    ProfScope ps(PK_TC_S4, s, 2.0 * M * N * K, 2.0 * (M * K + N * K) + 4.0 * M * N);
    fill_zero(y, sizeof(float) * (size_t)M4 * Dr, s);
    const __nv_bfloat16* A[3] = {T3, T3, T3};
    const __nv_bfloat16* B[3] = {Rb, Rb, Rb};
    const int p0[1] = {0};
    tc_gemm_bf16_pairs(A, ld3, B, ldr, M4, Dr, (int)K4, 1, p0, p0, y, Dr, tc::OUT_F32_ATOMIC,
                       s4_splitk(M4, Dr, kb), s, F.Rt ? &seg : nullptr);
  }
}

}  // namespace a2

namespace a2 {

// y = H_eff x with FP32-accurate tensor-core products: every BF16 GEMM operand is the
// three-plane split of an FP32/FP64 value and six plane pairs are accumulated in TMEM;
// the sparse MPO stages run in FP32.  L, R: three BF16 planes each (plane strides
// lplane / rplane elements, row strides ldl / ldr).  When A_{k+1} is folded, T2 is kept
// as three BF16 planes (the second K segment of S4 reads it through TMA).
void tc_heff_f32emu(cudaStream_t s, int n1, int n2, int Rl, int R1, int Rr, int Dl, int Dr,
                    const __nv_bfloat16* Lp, long long ldl, long long lplane,
                    const __nv_bfloat16* Rp, long long ldr, long long rplane, const double* x,
                    float* y, const SparseRows<float>& W1, const SparseRows<float>& W2,
                    const HeffFold& F, DevBuf& t1, DevBuf& t2, DevBuf& xa, DevBuf& tf) {
  static const int pa[6] = {0, 0, 1, 0, 1, 2};
  static const int pb[6] = {0, 1, 0, 2, 1, 0};
  const long long NX = (long long)n1 * n2 * Dr;
  const long long ldx = pad8(Dl);
  const long long xplane = NX * ldx;
  const long long s1 = (long long)Dl * Rl * NX;
  const long long s2 = (long long)Dl * R1 * NX;
  const long long p2 = (s2 + 63) / 64 * 64;          // T2 plane stride (split form)
  const long long K4 = (long long)Rr * Dr;
  const long long ld3 = pad8(K4);
  const long long M4 = (long long)Dl * n1 * n2;
  const long long plane3 = M4 * ld3;
  const bool t2split = F.Rt != nullptr;
  xa.ensure(sizeof(__nv_bfloat16) * (size_t)(3 * xplane), s);
  t1.ensure(std::max(sizeof(float) * (size_t)s1, sizeof(__nv_bfloat16) * (size_t)(3 * plane3)), s);
  t2.ensure(t2split ? sizeof(__nv_bfloat16) * (size_t)(3 * p2) : sizeof(float) * (size_t)s2, s);
  __nv_bfloat16* XT = xa.as<__nv_bfloat16>();
  float* T1 = t1.as<float>();
  float* T2 = t2.as<float>();
  __nv_bfloat16* T2p = t2.as<__nv_bfloat16>();
  __nv_bfloat16* T3 = t1.as<__nv_bfloat16>();
  // with both cores folded the S1-fold product needs its own FP32 buffer
  float* Tg = nullptr;
  if (F.Lt && t2split) {
    tf.ensure(sizeof(float) * (size_t)s2, s);
    Tg = tf.as<float>();
  }
  transpose_split3(x, Dl, (int)NX, XT, ldx, xplane, s);
  {  // S1
    const __nv_bfloat16* A[3] = {Lp, Lp + lplane, Lp + 2 * lplane};
    const __nv_bfloat16* B[3] = {XT, XT + xplane, XT + 2 * xplane};
    const double M = (double)Dl * Rl, N = (double)NX, K = Dl;
    ProfScope ps(PK_EMU_S1, s, 6.0 * 2.0 * M * N * K, 6.0 * (M * K + N * K) + 4.0 * M * N);
    tc_gemm_bf16_pairs(A, ldl, B, ldx, Dl * Rl, (int)NX, Dl, 6, pa, pb, T1, NX, tc::OUT_F32, 1, s);
  }
  if (F.Lt) {   // folded G of A_k: Lt x, FP32 (into T2, or into Tg when T2 is split)
    const __nv_bfloat16* A[3] = {F.Lt, F.Lt + F.ltplane, F.Lt + 2 * F.ltplane};
    const __nv_bfloat16* B[3] = {XT, XT + xplane, XT + 2 * xplane};
    const double M = (double)Dl * R1, N = (double)NX, K = Dl;
    ProfScope ps(PK_EMU_S1, s, 6.0 * 2.0 * M * N * K, 6.0 * (M * K + N * K) + 4.0 * M * N);
    tc_gemm_bf16_pairs(A, ldl, B, ldx, Dl * R1, (int)NX, Dl, 6, pa, pb, Tg ? Tg : T2, NX,
                       tc::OUT_F32, 1, s);
  }
  {  // S2 (FP32; W_rest added to the folded part when A_k is folded)
    ProfScope ps(PK_EMU_S2, s, 2.0 * W1.nnz_total * (double)n2 * Dr * Dl,
                 4.0 * (double)(s1 + s2) * (F.Lt ? 1.5 : 1.0));
    SparseGeom gm;
    gm.veclen = n2 * Dr;
    gm.in_sw = NX; gm.in_st = (long long)n2 * Dr;
    gm.out_sw = NX; gm.out_ss = (long long)n2 * Dr;
    gm.B1 = Dl; gm.in_b1 = (long long)Rl * NX; gm.out_b1 = (long long)R1 * NX;
    if (t2split) {
      sparse_rows_apply_split3<float, float>(W1, gm, T1, 0, Tg, T2p, p2, s);
    } else {
      gm.accumulate = F.Lt ? 1 : 0;
      sparse_rows_apply<float, float, float>(W1, gm, T1, T2, s);
    }
  }
  {  // S3 (FP32 or split input, three BF16 planes out)
    ProfScope ps(PK_EMU_S3, s, 2.0 * W2.nnz_total * (double)Dr * Dl * n1,
                 (t2split ? 6.0 : 4.0) * (double)s2 + 6.0 * (double)M4 * K4);
    SparseGeom gm;
    gm.veclen = Dr;
    gm.in_sw = NX; gm.in_st = Dr;
    gm.out_sw = Dr; gm.out_ss = ld3;
    gm.B1 = Dl; gm.B2 = n1;
    gm.in_b1 = (long long)R1 * NX; gm.in_b2 = (long long)n2 * Dr;
    gm.out_b1 = (long long)n1 * n2 * ld3; gm.out_b2 = (long long)n2 * ld3;
    if (t2split)
      sparse_rows_apply_split3<__nv_bfloat16, float>(W2, gm, T2p, p2, nullptr, T3, plane3, s);
    else
      sparse_rows_apply_split3<float, float>(W2, gm, T2, 0, nullptr, T3, plane3, s);
  }
  {  // S4 (+ the folded G of A_{k+1} as a second K segment over T2)
    const __nv_bfloat16* A[3] = {T3, T3 + plane3, T3 + 2 * plane3};
    const __nv_bfloat16* B[3] = {Rp, Rp + rplane, Rp + 2 * rplane};
    TcSeg2 seg;
    long long kb = (K4 + 63) / 64;
    if (t2split) {
      for (int i = 0; i < 3; ++i) {
        seg.A[i] = T2p + i * p2;
        seg.B[i] = F.Rt + i * F.rtplane;
      }
      seg.Dl = Dl; seg.n12 = n1 * n2; seg.R1 = R1; seg.Dr = Dr; seg.Nb = Dr;
      kb += (long long)R1 * ((Dr + 63) / 64);
    }
    const double M = (double)M4, N = Dr, K = (double)K4 + (t2split ? (double)R1 * Dr : 0.0);
    ProfScope ps(PK_EMU_S4, s, 6.0 * 2.0 * M * N * K, 6.0 * (M * K + N * K) + 4.0 * M * N);
    fill_zero(y, sizeof(float) * (size_t)M4 * Dr, s);
    tc_gemm_bf16_pairs(A, ld3, B, ldr, (int)M4, Dr, (int)K4, 6, pa, pb, y, Dr,
                       tc::OUT_F32_ATOMIC, s4_splitk(M4, Dr, kb), s,
                       t2split ? &seg : nullptr);
  }
}


// One-site H_eff with FP32-accurate tensor-core products (the one-site case of Alg. 2):
// T1 = L x (as S1), T2 = the MPO core on the rows in FP32 with three BF16 output planes
// (as S3), y = T2 R^T (as S4).
void tc_heff1_f32emu(cudaStream_t s, int n, int Rl, int Rr, int Dl, int Dr,
                     const __nv_bfloat16* Lp, long long ldl, long long lplane,
                     const __nv_bfloat16* Rp, long long ldr, long long rplane, const double* x,
                     float* y, const SparseRows<float>& W, DevBuf& t1, DevBuf& t2, DevBuf& xa) {
  static const int pa[6] = {0, 0, 1, 0, 1, 2};
  static const int pb[6] = {0, 1, 0, 2, 1, 0};
  const long long NX = (long long)n * Dr;
  const long long ldx = pad8(Dl);
  const long long xplane = (NX * ldx + 63) / 64 * 64;
  const long long s1 = (long long)Dl * Rl * NX;
  const long long K4 = (long long)Rr * Dr;
  const long long ld3 = pad8(K4);
  const long long M4 = (long long)Dl * n;
  const long long plane3 = (M4 * ld3 + 63) / 64 * 64;
  xa.ensure(sizeof(__nv_bfloat16) * (size_t)(3 * xplane), s);
  t1.ensure(sizeof(float) * (size_t)s1, s);
  t2.ensure(sizeof(__nv_bfloat16) * (size_t)(3 * plane3), s);
  __nv_bfloat16* XT = xa.as<__nv_bfloat16>();
  float* T1 = t1.as<float>();
  __nv_bfloat16* T2 = t2.as<__nv_bfloat16>();
  transpose_split3(x, Dl, (int)NX, XT, ldx, xplane, s);
  {
    const __nv_bfloat16* A[3] = {Lp, Lp + lplane, Lp + 2 * lplane};
    const __nv_bfloat16* B[3] = {XT, XT + xplane, XT + 2 * xplane};
    const double M = (double)Dl * Rl, N = (double)NX, K = Dl;
    ProfScope ps(PK_EMU_S1, s, 6.0 * 2.0 * M * N * K, 6.0 * (M * K + N * K) + 4.0 * M * N);
    tc_gemm_bf16_pairs(A, ldl, B, ldx, Dl * Rl, (int)NX, Dl, 6, pa, pb, T1, NX, tc::OUT_F32, 1, s);
  }
  {
    ProfScope ps(PK_EMU_S3, s, 2.0 * W.nnz_total * (double)Dr * Dl,
                 4.0 * (double)s1 + 6.0 * (double)M4 * K4);
    SparseGeom gm;
    gm.veclen = Dr;
    gm.in_sw = NX; gm.in_st = Dr;
    gm.out_sw = Dr; gm.out_ss = ld3;
    gm.B1 = Dl; gm.in_b1 = (long long)Rl * NX; gm.out_b1 = (long long)n * ld3;
    sparse_rows_apply_split3<float, float>(W, gm, T1, 0, nullptr, T2, plane3, s);
  }
  {
    const __nv_bfloat16* A[3] = {T2, T2 + plane3, T2 + 2 * plane3};
    const __nv_bfloat16* B[3] = {Rp, Rp + rplane, Rp + 2 * rplane};
    const double M = (double)M4, N = Dr, K = (double)K4;
    ProfScope ps(PK_EMU_S4, s, 6.0 * 2.0 * M * N * K, 6.0 * (M * K + N * K) + 4.0 * M * N);
    fill_zero(y, sizeof(float) * (size_t)M4 * Dr, s);
    tc_gemm_bf16_pairs(A, ld3, B, ldr, (int)M4, Dr, (int)K4, 6, pa, pb, y, Dr,
                       tc::OUT_F32_ATOMIC, s4_splitk(M4, Dr, (K4 + 63) / 64), s);
  }
}

// ============================================================================ FP64 emulation
// Ozaki scheme (Ozaki, Ogita, Oishi, Rump, "Error-free transformations of matrix
// multiplication by using fast routines of matrix multiplication and its applications",
// Numer. Algorithms 59, 2012) on the BF16 tensor cores.  Every row r of an FP64 operand
// is split into kOzSlices slices P_i[r][k] = q * 2^(e_r - kOzBits*i) with integer
// |q| <= 2^kOzBits - 1 (truncation of the remainder; e_r = ilogb(max_k |X[r][k]|) + 1),
// each exact in BF16.  A product of slice i of A with slice j of B is then an integer
// multiple of the unit 2^(e_r + e_c - kOzBits*(i+j)) of magnitude below 2^(2*kOzBits);
// all pairs of one level l = i + j share that unit, so a level's sum over at most
// 1024 / (l - 1) K indices per pair stays an integer below 2^24 units and the tensor
// cores' FP32 accumulation of it is exact.  The pairs with i + j <= kOzSlices + 1 are
// kept (the rest lie below 2^-kOzBits*kOzSlices of |A||B|), every level's tile of every K
// split is stored in FP32, and a combine kernel adds the tiles, smallest level first, with
// error-free two-sums into a pair of FP32 numbers (~2^-48 relative).
namespace {

// Slicing with integer operations only (the FP64 pipe is slow on this part): for a row
// with largest biased exponent field f_max, e = f_max - 1022 bounds |v| < 2^e; the
// fixed-point magnitude N = floor(|v| * 2^(56 - e)) < 2^56 is the significand shifted by
// f - e - 1019 bits, and slice i is bits [56 - 7i, 63 - 7i) of N times 2^(e - 7i) with the
// sign of v (the same digits as truncating the remainder slice by slice).  Scales below
// the FP32 normal range are flushed to zero.
static_assert(kOzSlices * kOzBits == 56, "the slices cover bits 0..55 of the fixed-point value");

__device__ __forceinline__ float pow2f(int k) {
  return (k >= -126 && k <= 127) ? __int_as_float((k + 127) << 23) : 0.f;
}

// One warp per row: the row's largest exponent by a warp reduction (no block barrier),
// then the slices of four consecutive entries per lane, each plane written as one 8-byte
// vector per lane (the kernel is bound by its 16 bytes of writes per entry).
// The 56-bit fixed-point magnitude of v at the row's scale 2^e (|v| < 2^e) and its sign.
__device__ __forceinline__ unsigned long long oz_fixed(double v, int e, float& sgn) {
  const long long bits = __double_as_longlong(v);
  int f = (int)((bits >> 52) & 0x7FF);
  unsigned long long m = (unsigned long long)bits & ((1ull << 52) - 1);
  if (f) m |= 1ull << 52;
  else f = 1;                                    // subnormal: no hidden bit
  const int sh = f - e - 1019;                   // <= 3 since |v| < 2^e
  sgn = bits < 0 ? -1.f : 1.f;
  return sh >= 0 ? (m << sh) : (sh > -64 ? (m >> -sh) : 0ull);
}
__global__ void __launch_bounds__(256)
ozaki_split_kernel(const double* __restrict__ X, long long sr, long long sk, int rows, int K,
                   __nv_bfloat16* __restrict__ P, long long ldp, long long plane) {
  const int lane = threadIdx.x & 31;
  const int nwarps = (int)((gridDim.x * blockDim.x) >> 5);
  for (int r = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); r < rows; r += nwarps) {
    const double* xr = X + (long long)r * sr;
    int fm = 0;
    for (int k = lane; k < K; k += 32)
      fm = max(fm, (int)((__double_as_longlong(xr[(long long)k * sk]) >> 52) & 0x7FF));
    for (int o = 16; o; o >>= 1) fm = max(fm, __shfl_xor_sync(0xffffffffu, fm, o));
    const int e = max(fm, 1) - 1022;
    __nv_bfloat16* pr = P + (long long)r * ldp;
    for (int k0 = 4 * lane; k0 < K; k0 += 128) {
      unsigned long long N[4];
      float sgn[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        sgn[u] = 1.f;
        N[u] = k0 + u < K ? oz_fixed(xr[(long long)(k0 + u) * sk], e, sgn[u]) : 0ull;
      }
#pragma unroll
      for (int i = 1; i <= kOzSlices; ++i) {
        const float sc = pow2f(e - kOzBits * i);
        float w[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int q = (int)((N[u] >> (56 - kOzBits * i)) & ((1u << kOzBits) - 1));
          w[u] = sgn[u] * (float)q * sc;   // exact in BF16
        }
        __nv_bfloat16* dst = pr + (long long)(i - 1) * plane + k0;
        if (k0 + 4 <= K) {   // ldp % 8 == 0, plane % 64 == 0, k0 % 4 == 0: 8-byte aligned
          const __nv_bfloat162 lo = __floats2bfloat162_rn(w[0], w[1]);
          const __nv_bfloat162 hi = __floats2bfloat162_rn(w[2], w[3]);
          uint2 pk;
          pk.x = *reinterpret_cast<const unsigned int*>(&lo);
          pk.y = *reinterpret_cast<const unsigned int*>(&hi);
          *reinterpret_cast<uint2*>(dst) = pk;
        } else {
          for (int u = 0; u < 4; ++u)
            if (k0 + u < K) dst[u] = __float2bfloat16_rn(w[u]);
        }
      }
    }
  }
}

// Slices of the rows of X^T, X a (K x N) row-major matrix (row stride ldx): output row n
// holds X[k][n], k < K.  A block takes 32 consecutive output rows: the exponent pass and
// the slicing read X row by row (coalesced across the 32 columns), the slices of a
// 64-wide K chunk are staged in shared memory and leave as 8-byte vectors along K.  Same
// slices as ozaki_split of the transposed matrix.
constexpr int kOzColChunk = 64, kOzColPad = kOzColChunk + 4;   // row of 68 BF16 = 136 B
__global__ void __launch_bounds__(256)
ozaki_split_cols_kernel(const double* __restrict__ X, long long ldx, int N, int K,
                        __nv_bfloat16* __restrict__ P, long long ldp, long long plane) {
  __shared__ int emax[8][32];
  __shared__ __align__(16) __nv_bfloat16 tile[kOzSlices][32][kOzColPad];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int n0 = blockIdx.x * 32, n = n0 + lane;
  int fm = 0;
  if (n < N)
    for (int k = warp; k < K; k += 8)
      fm = max(fm, (int)((__double_as_longlong(X[(long long)k * ldx + n]) >> 52) & 0x7FF));
  emax[warp][lane] = fm;
  __syncthreads();
  fm = 0;
#pragma unroll
  for (int w = 0; w < 8; ++w) fm = max(fm, emax[w][lane]);
  const int e = max(fm, 1) - 1022;
  for (int k0 = 0; k0 < K; k0 += kOzColChunk) {
#pragma unroll
    for (int t = 0; t < kOzColChunk / 8; ++t) {
      const int kk = warp + 8 * t, k = k0 + kk;
      float sgn = 1.f;
      const unsigned long long Nq =
          (n < N && k < K) ? oz_fixed(X[(long long)k * ldx + n], e, sgn) : 0ull;
#pragma unroll
      for (int i = 1; i <= kOzSlices; ++i) {
        const int q = (int)((Nq >> (56 - kOzBits * i)) & ((1u << kOzBits) - 1));
        tile[i - 1][lane][kk] = __float2bfloat16_rn(sgn * (float)q * pow2f(e - kOzBits * i));
      }
    }
    __syncthreads();
    // 8 slices x 32 rows x 16 vectors of 4 values
    for (int v = threadIdx.x; v < kOzSlices * 32 * (kOzColChunk / 4); v += blockDim.x) {
      const int i = v / (32 * (kOzColChunk / 4)), r = (v / (kOzColChunk / 4)) % 32;
      const int c4 = v % (kOzColChunk / 4), k = k0 + 4 * c4;
      if (n0 + r >= N || k >= K) continue;
      __nv_bfloat16* dst = P + (long long)i * plane + (long long)(n0 + r) * ldp + k;
      const __nv_bfloat16* src = &tile[i][r][4 * c4];
      if (k + 4 <= K)   // ldp % 8 == 0, plane % 64 == 0, k % 4 == 0: 8-byte aligned
        *reinterpret_cast<uint2*>(dst) = *reinterpret_cast<const uint2*>(src);
      else
        for (int u = 0; k + u < K; ++u) dst[u] = src[u];
    }
    __syncthreads();
  }
}

// C[r][c] = sum over the level tiles: tile t of level lev[t] at T + t * MN (row-major,
// N columns); tiles ordered by level (largest level last).
// C[r][c] = sum of all level tiles (tile t at T + t * MN, row-major with N columns,
// ordered by level, largest level last), added smallest level first in double-float
// arithmetic: every tile value is exact, the two-sum keeps the running sum as an FP32
// pair hi + lo (~2^-48), and the result is written as FP64 (hi + lo) or as the pair.
template <bool DF>
__global__ void ozaki_combine_kernel(const float* __restrict__ T, long long MN, int nt, int N,
                                     double* __restrict__ C, float* __restrict__ Cdf,
                                     long long df_plane, long long ldc) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < MN;
       e += (long long)gridDim.x * blockDim.x) {
    float hi = 0.f, lo = 0.f;
    for (int t = nt - 1; t >= 0; --t) {
      const float v = __ldg(T + (long long)t * MN + e);
      const float s = __fadd_rn(hi, v);
      const float bp = __fsub_rn(s, hi);
      const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(v, bp));
      hi = s;
      lo = __fadd_rn(lo, err);
    }
    const long long o = (e / N) * ldc + e % N;
    if constexpr (DF) {   // renormalised pair
      const float s = __fadd_rn(hi, lo);
      Cdf[o] = s;
      Cdf[df_plane + o] = __fsub_rn(lo, __fsub_rn(s, hi));
    } else {
      C[o] = (double)hi + (double)lo;
    }
  }
}

}  // namespace

void ozaki_split_cols(const double* X, long long ldx, int N, int K, __nv_bfloat16* P,
                      long long ldp, long long plane, cudaStream_t s) {
  if (N <= 0 || K <= 0) return;
  ozaki_split_cols_kernel<<<(N + 31) / 32, 256, 0, s>>>(X, ldx, N, K, P, ldp, plane);
  A2_CHECK_LAUNCH();
}

void ozaki_split(const double* X, long long sr, long long sk, int rows, int K, __nv_bfloat16* P,
                 long long ldp, long long plane, cudaStream_t s) {
  if (rows <= 0 || K <= 0) return;
  const int grid = std::min((rows + 7) / 8, 152 * 8);   // eight rows (warps) per block
  ozaki_split_kernel<<<grid, 256, 0, s>>>(X, sr, sk, rows, K, P, ldp, plane);
  A2_CHECK_LAUNCH();
}

void tc_gemm_f64emu(const __nv_bfloat16* A, long long lda, long long aplane,
                    const __nv_bfloat16* B, long long ldb, long long bplane, int M, int N, int K,
                    double* C, long long ldc, DevBuf& slab, cudaStream_t s, float* Cdf,
                    long long df_plane) {
  if (M <= 0 || N <= 0) return;
  static int num_sms = 0;
  static std::once_flag sms_once;
  std::call_once(sms_once, [] {
    int dev = 0;
    A2_CUDA(cudaGetDevice(&dev));
    A2_CUDA(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev));
  });
  const __nv_bfloat16* Ap[tc::kMaxPlanes];
  const __nv_bfloat16* Bp[tc::kMaxPlanes];
  for (int i = 0; i < tc::kMaxPlanes; ++i) {
    Ap[i] = A + i * aplane;
    Bp[i] = B + i * bplane;
  }
  // K splits: at most kOzSplitBlocks K blocks per split (bounds the number of chunk sums
  // per accumulator, hence the rounding of its lo part), and enough work units to fill
  // the GPU when the output has few tiles
  constexpr int kOzSplitBlocks = 64;
  const int nk = (K + tc::BK - 1) / tc::BK;
  const long long tiles = (long long)cdiv(M, tc::BM) * cdiv(N, tc::kOzBN);
  int splits = cdiv(nk, kOzSplitBlocks);
  if (tiles < num_sms) splits = std::max<int>(splits, (int)cdiv(2LL * num_sms, tiles));
  splits = std::max(1, std::min(splits, nk));
  splits = cdiv(nk, cdiv(nk, splits));   // the count launch_oz will use
  if (splits == 1) {
    if (Cdf) tc::launch_oz(Ap, lda, Bp, ldb, M, N, K, 1, tc::OZ_PAIR, Cdf, ldc, df_plane, s);
    else tc::launch_oz(Ap, lda, Bp, ldb, M, N, K, 1, tc::OZ_F64, C, ldc, 0, s);
    return;
  }
  const long long MN = (long long)M * N;
  slab.ensure(sizeof(float) * (size_t)(2LL * splits * MN), s);
  float* T = slab.as<float>();
  tc::launch_oz(Ap, lda, Bp, ldb, M, N, K, splits, tc::OZ_SPLIT, T, N, 0, s);
  const int grid = (int)std::min<long long>((MN + 255) / 256, 152LL * 16);
  if (Cdf)
    ozaki_combine_kernel<true><<<grid, 256, 0, s>>>(T, MN, 2 * splits, N, nullptr, Cdf,
                                                    df_plane, ldc);
  else
    ozaki_combine_kernel<false><<<grid, 256, 0, s>>>(T, MN, 2 * splits, N, C, nullptr, 0, ldc);
  A2_CHECK_LAUNCH();
}

}  // namespace a2
