// Kernel bodies as operations. An operation is a struct with an argument record
// `Args` and a device body `run<PS>(ctx, args)` that does the work of one block
// of its launch grid. A plain kernel launch runs the body once per hardware
// block (ctx = blockIdx.x of gridDim.x). The persistent executor (persist.cu)
// replays recorded launches inside one cooperative kernel, where every CTA runs
// the bodies of some virtual blocks of each launch in turn; there PS = true and
// loads of vectors that earlier launches of the same kernel wrote go through L2
// (ld.global.cg), because L1 is not coherent across SMs within one kernel.
//
// Recording: while a Recorder is active on the calling host thread, launch_op
// appends (operation id, grid, block, shared memory, argument record) to it
// instead of launching.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstring>
#include <type_traits>
#include <vector>

namespace fde {

void note_launches(int n);

// Block index and grid size of the body's launch (virtual inside the executor).
struct Ctx {
  long long bid, nblk;
};
__device__ __forceinline__ Ctx hw_ctx() { return Ctx{(long long)blockIdx.x, (long long)gridDim.x}; }

// Load of data that may have been written earlier in the same kernel (PS).
template <bool PS, typename T> __device__ __forceinline__ T ldv(const T* p) {
  if constexpr (PS) return __ldcg(p);
  else return *p;
}

// Threads per block of every recorded launch (the executor's CTA size).
constexpr int kPersistThreads = 256;
// Bytes of one recorded command: a 32-byte header and the argument record.
constexpr int kCmdBytes = 512;
constexpr int kCmdHeaderBytes = 32;
constexpr int kCmdArgBytes = kCmdBytes - kCmdHeaderBytes;

struct CmdHeader {
  int op;             // index of the operation in PersistOps
  unsigned grid;      // blocks of the launch
  unsigned smem;      // dynamic shared memory of a block
  int threads;        // threads of a block (kPersistThreads)
  const void* kernel; // the operation's named kernel (host stub; stream replay)
  long long pad;
};
static_assert(sizeof(CmdHeader) == kCmdHeaderBytes, "command header layout");

struct Recorder {
  std::vector<unsigned char> cmds;  // kCmdBytes per command
  size_t max_smem = 0;
  int error = 0;  // 1: a launch that the executor cannot run was requested
  long long count() const { return (long long)(cmds.size() / kCmdBytes); }
};

// The recorder of the calling host thread (null: launches run).
Recorder*& active_recorder();
inline bool recording() { return active_recorder() != nullptr; }

template <class... Ops> struct OpList {};

template <class Op, class List> struct OpIndex;
template <class Op> struct OpIndex<Op, OpList<>> { static constexpr int value = -1; };
template <class Op, class H, class... T> struct OpIndex<Op, OpList<H, T...>> {
  static constexpr int tail = OpIndex<Op, OpList<T...>>::value;
  static constexpr int value = std::is_same<Op, H>::value ? 0 : (tail < 0 ? -1 : 1 + tail);
};

// Launch `kern` (the operation's named kernel) or record the launch.
template <class Op, class PersistList>
cudaError_t launch_or_record(void (*kern)(typename Op::Args), unsigned grid, int threads, size_t smem,
                             cudaStream_t st, const typename Op::Args& a) {
  static_assert(std::is_trivially_copyable<typename Op::Args>::value, "argument records are copied bytewise");
  static_assert(sizeof(typename Op::Args) <= kCmdArgBytes, "argument record larger than a command");
  if (Recorder* r = active_recorder()) {
    constexpr int id = OpIndex<Op, PersistList>::value;
    if (id < 0 || threads != kPersistThreads || grid == 0) {
      r->error = 1;
      return cudaSuccess;
    }
    const size_t at = r->cmds.size();
    r->cmds.resize(at + kCmdBytes, 0);
    CmdHeader h{id, grid, (unsigned)smem, threads, reinterpret_cast<const void*>(kern), 0};
    std::memcpy(r->cmds.data() + at, &h, sizeof(h));
    std::memcpy(r->cmds.data() + at + kCmdHeaderBytes, &a, sizeof(a));
    if (smem > r->max_smem) r->max_smem = smem;
    return cudaSuccess;
  }
  kern<<<grid, threads, smem, st>>>(a);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace fde
