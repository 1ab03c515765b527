// Inline-PTX helpers for sm_103a: mbarriers with bounded waits and the
// untiled bulk (TMA) copy global -> shared.  No multicast form is used.
#pragma once
#include <cstdint>

namespace dd {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// End a barrier object's life (no thread waits on it, nothing arrives on it any more).
__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Arrive once on the barrier and add `bytes` to its expected transaction count.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// Plain arrival (count 1) on the barrier.
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

// Non-blocking test: has phase `parity` of the barrier completed?
__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

// Wait for phase `parity` of the barrier to complete, giving up after
// `limit_cycles` SM clock cycles (returns false then).  Every wait in this
// library is bounded so that a lost copy becomes an error status, not a hang.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, long long limit_cycles) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long start = clock64();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (clock64() - start > limit_cycles) return false;
  }
}

// 1-D bulk copy of `bytes` (multiple of 16) from global `src` (16-B aligned)
// into shared `dst` (16-B aligned); completion is signalled on `bar` as
// transaction bytes.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// About one second at GB300 clocks.
constexpr long long kWaitLimitCycles = 2000000000LL;

// Device-side error codes written to the plan's status word.
enum DeviceError : int { kDevOk = 0, kDevWaitTimeout = 1, kDevBadDescriptor = 2, kDevBadIndex = 3 };

__device__ __forceinline__ void report_error(int* status, int code) {
  if (status) atomicCAS(status, 0, code);
}

// Checked builds (-DDD_CHECKED, used by the tests as a sanitizer stand-in):
// an index outside its buffer records kDevBadIndex in the status word and the
// caller skips the access; in normal builds the check compiles away.
__device__ __forceinline__ bool index_ok(int* status, bool cond) {
  if (!cond) report_error(status, kDevBadIndex);
  return cond;
}
#ifdef DD_CHECKED
#define DD_INDEX_OK(status, cond) ::dd::index_ok((status), (cond))
#else
#define DD_INDEX_OK(status, cond) true
#endif

}  // namespace dd

// ---------------------------------------------------------------- tcgen05
// Tensor Memory (TMEM) used as a per-lane scratch row: a warp may access the
// 32 TMEM lanes of its quadrant (warp % 4); an address is (lane << 16) | column.
namespace dd {

// Allocate `ncols` columns (power of two, 32..512) for this CTA; warp-wide.
// The base address is written to shared memory at `dst`.
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
// Free an allocation; warp-wide, by the warp that allocated it.
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tmem_fence_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tmem_fence_after_sync() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Each thread loads 32 consecutive 32-bit columns of its own lane.
// Two independent fp32 additions, a_k + b_k rounded to nearest, in one
// instruction; each lane's result is the scalar add's bit for bit.
__device__ __forceinline__ void add2_rn(float& a0, float& a1, float b0, float b1) {
  asm("{\n .reg .b64 x, y;\n mov.b64 x, {%0, %1};\n mov.b64 y, {%2, %3};\n add.rn.f32x2 x, x, y;\n"
      " mov.b64 {%0, %1}, x;\n}\n"
      : "+f"(a0), "+f"(a1)
      : "f"(b0), "f"(b1));
}

// Two independent fused multiply-adds, w * b_k + a_k with one rounding each,
// in one instruction; each lane's result is fmaf's bit for bit.
__device__ __forceinline__ void fma2_rn(float& a0, float& a1, float w, float b0, float b1) {
  asm("{\n .reg .b64 x, y, s;\n mov.b64 x, {%0, %1};\n mov.b64 y, {%2, %3};\n mov.b64 s, {%4, %4};\n"
      " fma.rn.f32x2 x, s, y, x;\n mov.b64 {%0, %1}, x;\n}\n"
      : "+f"(a0), "+f"(a1)
      : "f"(b0), "f"(b1), "f"(w));
}

// Two independent fused multiply-adds of pairs, x_k * y_k + a_k with one
// rounding each, in one instruction; each lane's result is fmaf's bit for bit.
__device__ __forceinline__ void fma2v_rn(float& a0, float& a1, float x0, float x1, float y0, float y1) {
  asm("{\n .reg .b64 a, x, y;\n mov.b64 a, {%0, %1};\n mov.b64 x, {%2, %3};\n mov.b64 y, {%4, %5};\n"
      " fma.rn.f32x2 a, x, y, a;\n mov.b64 {%0, %1}, a;\n}\n"
      : "+f"(a0), "+f"(a1)
      : "f"(x0), "f"(x1), "f"(y0), "f"(y1));
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
      "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7]), "=f"(v[8]),
        "=f"(v[9]), "=f"(v[10]), "=f"(v[11]), "=f"(v[12]), "=f"(v[13]), "=f"(v[14]), "=f"(v[15]), "=f"(v[16]),
        "=f"(v[17]), "=f"(v[18]), "=f"(v[19]), "=f"(v[20]), "=f"(v[21]), "=f"(v[22]), "=f"(v[23]), "=f"(v[24]),
        "=f"(v[25]), "=f"(v[26]), "=f"(v[27]), "=f"(v[28]), "=f"(v[29]), "=f"(v[30]), "=f"(v[31])
      : "r"(taddr)
      : "memory");
}

// Each thread loads 16 consecutive 32-bit columns of its own lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7]), "=f"(v[8]),
        "=f"(v[9]), "=f"(v[10]), "=f"(v[11]), "=f"(v[12]), "=f"(v[13]), "=f"(v[14]), "=f"(v[15])
      : "r"(taddr));
}

// Wait for this thread's Tensor Memory loads, naming the 16 registers the
// last load wrote as operands, so that no use of them can be scheduled
// before the wait.
__device__ __forceinline__ void tmem_wait_ld16(float* v) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+f"(v[0]), "+f"(v[1]), "+f"(v[2]), "+f"(v[3]), "+f"(v[4]), "+f"(v[5]), "+f"(v[6]), "+f"(v[7]),
                 "+f"(v[8]), "+f"(v[9]), "+f"(v[10]), "+f"(v[11]), "+f"(v[12]), "+f"(v[13]), "+f"(v[14]),
                 "+f"(v[15])
               :
               : "memory");
}

// Four 16-byte chunks of this thread's lane to 16 consecutive columns.
__device__ __forceinline__ void tmem_st16(uint32_t taddr, float4 x0, float4 x1, float4 x2, float4 x3) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
          taddr),
      "f"(x0.x), "f"(x0.y), "f"(x0.z), "f"(x0.w), "f"(x1.x), "f"(x1.y), "f"(x1.z), "f"(x1.w), "f"(x2.x), "f"(x2.y),
      "f"(x2.z), "f"(x2.w), "f"(x3.x), "f"(x3.y), "f"(x3.z), "f"(x3.w));
}
}  // namespace dd

// -------------------------------------------------------------- TMA tiles
namespace dd {

// 3-D tiled TMA load (coordinates innermost first) into shared memory,
// completion as transaction bytes on `bar`.
__device__ __forceinline__ void tma_load_3d(void* dst, const void* tmap, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

// Bring a tensor map (generic address of global, constant or kernel
// parameter memory) into the TMA unit's descriptor cache ahead of its first use.
__device__ __forceinline__ void prefetch_tensormap(const void* tmap) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(tmap)) : "memory");
}

}  // namespace dd
