// Persistent executor of recorded launches.
//
// A recorded launch (op.cuh) is an operation id, a grid, a block size (256), the
// operation's named kernel and an argument record. Replaying it means running the operation's body for every
// block index of its grid; a kernel boundary between two launches is replaced by
// a barrier of the CTAs that ran them. The executor is one cooperative kernel
// (all CTAs resident): its CTAs are split into instance groups of equal size;
// the first CTA of a group takes the next instance from a device-side queue and
// the whole group runs that instance's launches in their recorded order, the
// blocks of each launch spread over the group's CTAs (virtual block b on CTA
// b mod group size), with a group barrier after each launch. Instances are
// independent, so groups never wait on each other.
//
// Lockstep schedule: when every instance recorded the same number of launches
// (the batch solve's fixed budgets make the sequences alike), step k runs launch
// k of every instance at once: the blocks of those launches form one index
// space (prefix sums of their grids), spread over all CTAs, followed by one
// barrier of all CTAs. This balances instances of very different sizes across
// the whole GPU.
//
// Barrier: each CTA's thread 0 fences its block's writes (after a block-wide
// __syncthreads), adds one to the group's arrival counter and spins with an
// acquire load until the counter reaches the CTA's own count of arrivals
// expected so far. Every spin is bounded by a %globaltimer deadline; a spin that
// runs out records FDE_ETIMEOUT (with the group and the last finished command)
// and its CTA returns; any CTA that sees a recorded failure while waiting
// returns too, so the kernel ends within about one more limit.
#include "ops_fft.cuh"
#include "ops_prec_reg.cuh"
#include "ops_vec.cuh"
#include "persist.h"
#include "toeplitz_reg.cuh"

namespace fde {

Recorder*& active_recorder() {
  static thread_local Recorder* r = nullptr;
  return r;
}

// One operation's body as a separate (not inlined) function: each body keeps
// its own register allocation instead of one allocation for all of them. The
// body works on a private copy of its argument record: the body's stores to
// global memory could alias the record where it lies, which would make the
// compiler reload its fields after every store.
template <class Op> __device__ __noinline__ void run_persistent(const Ctx& c, const unsigned char* args) {
  using A = typename Op::Args;
  static_assert(sizeof(A) % 8 == 0 && alignof(A) <= 8, "argument records are copied in 8-byte words");
  unsigned long long w[sizeof(A) / 8];
  const unsigned long long* src = reinterpret_cast<const unsigned long long*>(args);
#pragma unroll
  for (int i = 0; i < (int)(sizeof(A) / 8); ++i) w[i] = __ldg(src + i);
  Op::template run<true>(c, *reinterpret_cast<const A*>(w));
}

template <class List> struct Exec;
template <class... Ops> struct Exec<OpList<Ops...>> {
  // body of command `op` for virtual block c.bid; args point to its argument record
  __device__ static void run(int op, const Ctx& c, const unsigned char* args) {
    int i = 0;
    (void)((op == i++ ? (run_persistent<Ops>(c, args), true) : false) || ...);
  }
};
using PersistExec = Exec<PersistOps>;

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ long long ld_acquire(const long long* p) {
  long long v;
  asm volatile("ld.acquire.gpu.global.s64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// Per-CTA state of the group barrier (used by thread 0).
struct GroupBarrier {
  unsigned* counter;
  unsigned expected;  // arrivals of the whole group so far, this CTA's count
  int size;
  bool skip_next;     // test hook: do not arrive at the next barrier
};

// Returns false (in every thread of the block) when the wait ran out or another
// CTA recorded a failure; the caller then returns from the kernel.
__device__ bool group_sync(GroupBarrier& b, const PersistLaunch& pl, int group, long long done) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    b.expected += (unsigned)b.size;
    __threadfence();
    if (!b.skip_next) atomicAdd(b.counter, 1u);
    b.skip_next = false;
    int ok = 1;
    const unsigned long long t0 = global_ns();
    while ((int)(ld_acquire(b.counter) - b.expected) < 0) {
      if (ld_acquire(pl.status) != 0) {
        ok = 0;
        break;
      }
      if (global_ns() - t0 > pl.timeout_ns) {
        if (atomicCAS(reinterpret_cast<unsigned long long*>(pl.status), 0ull,
                      (unsigned long long)(long long)FDE_ETIMEOUT) == 0ull) {
          pl.status[1] = group;
          pl.status[2] = done;
        }
        ok = 0;
        break;
      }
      __nanosleep(64);
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

__global__ void __launch_bounds__(kPersistThreads, 2) k_persist(PersistLaunch pl) {
  __shared__ int s_inst;
  const int g = blockIdx.x / pl.group_ctas, rank = blockIdx.x - g * pl.group_ctas;
  if (g >= pl.groups) return;
  GroupBarrier bar{pl.bar + g, 0u, pl.group_ctas, pl.stall_group == g && rank == 0};
  long long done = -1;  // last finished command (global index)
  for (;;) {
    if (rank == 0 && threadIdx.x == 0) {
      const int q = atomicAdd(pl.queue, 1);
      pl.slot[g] = q < pl.count ? pl.order[q] : -1;
    }
    if (!group_sync(bar, pl, g, done)) return;
    if (threadIdx.x == 0) s_inst = __ldcg(pl.slot + g);
    __syncthreads();
    const int inst = s_inst;
    if (inst < 0) return;
    const long long c1 = pl.off[inst + 1];
    for (long long k = pl.off[inst]; k < c1; ++k) {
      const unsigned char* cmd = pl.cmds + k * kCmdBytes;
      const CmdHeader h = *reinterpret_cast<const CmdHeader*>(cmd);
      for (long long vb = rank; vb < (long long)h.grid; vb += pl.group_ctas)
        PersistExec::run(h.op, Ctx{vb, (long long)h.grid}, cmd + kCmdHeaderBytes);
      done = k;
      if (!group_sync(bar, pl, g, done)) return;
    }
  }
}

__global__ void __launch_bounds__(kPersistThreads, 2) k_persist_lockstep(PersistLaunch pl) {
  GroupBarrier bar{pl.bar, 0u, (int)gridDim.x, pl.stall_group == 0 && blockIdx.x == 0};
  const int n = pl.count;
  for (int k = 0; k < pl.steps; ++k) {
    const int* pre = pl.vstart + (long long)k * (n + 1);
    const long long V = pre[n];
    for (long long vb = blockIdx.x; vb < V; vb += gridDim.x) {
      int lo = 0, hi = n;  // largest i with pre[i] <= vb
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (pre[mid] <= vb) lo = mid;
        else hi = mid;
      }
      const unsigned char* cmd = pl.cmds + (pl.off[lo] + k) * kCmdBytes;
      const CmdHeader h = *reinterpret_cast<const CmdHeader*>(cmd);
      PersistExec::run(h.op, Ctx{vb - pre[lo], (long long)h.grid}, cmd + kCmdHeaderBytes);
    }
    if (!group_sync(bar, pl, 0, k)) return;
  }
}

cudaError_t persist_prepare(size_t smem, int* ctas_per_sm) {
  cudaError_t e = cudaFuncSetAttribute(k_persist_lockstep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_persist, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int a = 0, b = 0;
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_persist, kPersistThreads, smem);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_persist_lockstep, kPersistThreads, smem);
  *ctas_per_sm = a < b ? a : b;
  return e;
}

cudaError_t persist_run(const PersistLaunch& pl, size_t smem, cudaStream_t st) {
  PersistLaunch a = pl;
  void* args[] = {&a};
  const void* kern = pl.steps > 0 ? (const void*)k_persist_lockstep : (const void*)k_persist;
  const cudaError_t e = cudaLaunchCooperativeKernel(kern, dim3((unsigned)(pl.groups * pl.group_ctas)),
                                                    dim3(kPersistThreads), args, smem, st);
  note_launches(1);
  return e;
}

cudaError_t persist_replay(const unsigned char* cmds, long long n, cudaStream_t st) {
  for (long long k = 0; k < n; ++k) {
    CmdHeader h;
    std::memcpy(&h, cmds + k * kCmdBytes, sizeof(h));
    void* args[] = {const_cast<unsigned char*>(cmds + k * kCmdBytes + kCmdHeaderBytes)};
    const cudaError_t e = cudaLaunchKernel(h.kernel, dim3(h.grid), dim3(h.threads), args, h.smem, st);
    if (e != cudaSuccess) return e;
  }
  note_launches((int)n);
  return cudaSuccess;
}

}  // namespace fde
