// Host <-> device transfers of the host-buffer entry points. Pinned host memory
// (cudaHostAlloc / cudaHostRegister) is mapped into the device's address space,
// so a kernel reads or writes it directly over the CPU-GPU link: the SMs move
// the data instead of the copy engines, whose transfers measured 3-8x slower
// right after a long solve (58-68 GB/s out, 26 GB/s in, against 192 and 210 GB/s
// for the kernel). Pageable host memory, and device memory of another GPU, go
// through cudaMemcpyAsync.
#include "internal.h"

namespace fde {

namespace {

// dst[i] = src[i]; 16-byte accesses when both arrays allow them
__global__ void k_copy_f64(const double* __restrict__ src, double* __restrict__ dst, long long n, int vec2) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long i0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (vec2) {
    const long long n2 = n / 2;
    const double2* s2 = reinterpret_cast<const double2*>(src);
    double2* d2 = reinterpret_cast<double2*>(dst);
    for (long long i = i0; i < n2; i += stride) d2[i] = s2[i];
    if (i0 == 0 && (n & 1)) dst[n - 1] = src[n - 1];
  } else {
    for (long long i = i0; i < n; i += stride) dst[i] = src[i];
  }
}

// The device address of a host buffer: pinned memory maps to an address the
// kernel can use; pageable memory has none (*mapped = false).
cudaError_t device_address(const void* host, const void** dev, bool* mapped) {
  cudaPointerAttributes at{};
  cudaError_t e = cudaPointerGetAttributes(&at, host);
  if (e != cudaSuccess) return e;
  if (at.type == cudaMemoryTypeHost) {
    void* d = nullptr;
    if ((e = cudaHostGetDevicePointer(&d, const_cast<void*>(host), 0)) != cudaSuccess) return e;
    *dev = d;
    *mapped = true;
  } else if (at.type == cudaMemoryTypeManaged) {
    *dev = host;
    *mapped = true;
  } else if (at.type == cudaMemoryTypeDevice) {
    // device memory of this GPU is used in place; another GPU's memory is not
    // addressable by this GPU's kernels without peer access, so it goes through
    // cudaMemcpyAsync (cudaMemcpyDefault resolves the direction by address)
    int cur = -1;
    if ((e = cudaGetDevice(&cur)) != cudaSuccess) return e;
    *dev = at.device == cur ? host : nullptr;
    *mapped = at.device == cur;
  } else {
    *dev = nullptr;
    *mapped = false;
  }
  return cudaSuccess;
}

cudaError_t copy_kernel(double* dst, const double* src, long long n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int vec2 = ((uintptr_t)dst % 16 == 0) && ((uintptr_t)src % 16 == 0);
  long long g = ((vec2 ? n / 2 : n) + 255) / 256;
  if (g > 152LL * 8) g = 152LL * 8;
  if (g < 1) g = 1;
  k_copy_f64<<<(unsigned)g, 256, 0, st>>>(src, dst, n, vec2);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace

cudaError_t copy_from_host(double* dev_dst, const double* host_src, long long n, cudaStream_t st) {
  const void* src = nullptr;
  bool mapped = false;
  cudaError_t e = device_address(host_src, &src, &mapped);
  if (e != cudaSuccess) return e;
  if (mapped) return copy_kernel(dev_dst, static_cast<const double*>(src), n, st);
  return cudaMemcpyAsync(dev_dst, host_src, sizeof(double) * n, cudaMemcpyDefault, st);
}

cudaError_t copy_to_host(double* host_dst, const double* dev_src, long long n, cudaStream_t st) {
  const void* dst = nullptr;
  bool mapped = false;
  cudaError_t e = device_address(host_dst, &dst, &mapped);
  if (e != cudaSuccess) return e;
  if (mapped) return copy_kernel(static_cast<double*>(const_cast<void*>(dst)), dev_src, n, st);
  return cudaMemcpyAsync(host_dst, dev_src, sizeof(double) * n, cudaMemcpyDefault, st);
}

}  // namespace fde
