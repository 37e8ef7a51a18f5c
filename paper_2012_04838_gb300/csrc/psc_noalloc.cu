// Shell spectra without any device allocation.
//
// Some callers cannot call cudaMalloc or hand the library a workspace: code
// running inside a CUDA-graph-replayed pipeline whose memory is fixed up front,
// plugins hosted by an application that owns the device allocator, or tools that
// only hold a pointer to an existing state.  For them this file provides a
// variant of the shell-spectrum reduction whose per-shell partial sums live in
// a file-scope device array instead of the simulation workspace.
//
// The array is sized for PSC_NOALLOC_MAX_SHELLS shells (40 KB of FP64 sums) and,
// like every __device__ variable, occupies that memory on every GPU that loads
// the library until the process exits.
#include <mutex>
#include <string>

#include "psc.h"
// only the (template) shell reduction; the other kernels live in psc_capi.cu
#define PSC_SHELLS_ONLY
#include "psc_kernels.cuh"

namespace {

constexpr int kMaxShells = PSC_NOALLOC_MAX_SHELLS;
constexpr int kMaxDevices = 64;

// Scratch shared by every call on a device: raw per-shell sums of the last call.
static __device__ __align__(256) double g_shell_scratch[psc::NSQ * kMaxShells];

std::mutex g_setup_mu;
double* g_scratch_ptr[kMaxDevices] = {};  // device address of g_shell_scratch, per device

// E(n) = raw_u(n) / (2 N^6), E_phi(n) = raw_phi(n) / (2 N^6)
__global__ void k_noalloc_finish(const double* raw, int nshell, double inv2n6, double* Ek, double* Ephi) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nshell) return;
  Ek[n] = raw[n] * inv2n6;
  Ephi[n] = raw[nshell + n] * inv2n6;
}

int shells_for(int N) {
  const int K = (N - 1) / 3;
  int n = 0;
  while ((long long)(n + 1) * (n + 1) - (n + 1) < 3LL * K * K) ++n;  // largest shell holding |k|^2 = 3K^2
  return n + 1;
}

}  // namespace

namespace psc {
void set_error(const std::string& msg);
}

extern "C" psc_status psc_shell_spectra_noalloc(const void* state, int32_t N, int32_t precision, double* Ek,
                                                double* Ephi, int32_t nshell_cap, void* stream) {
  if (!state || !Ek || !Ephi) {
    psc::set_error("psc_shell_spectra_noalloc: null pointer");
    return PSC_EINVAL;
  }
  if (N < 8 || (precision != PSC_FP64 && precision != PSC_FP32_MIXED)) {
    psc::set_error("psc_shell_spectra_noalloc: N must be >= 8 and precision PSC_FP64 or PSC_FP32_MIXED");
    return PSC_EINVAL;
  }
  const int nshell = shells_for(N);
  if (nshell > kMaxShells) {
    psc::set_error("psc_shell_spectra_noalloc: N=" + std::to_string(N) + " needs " + std::to_string(nshell) +
                   " shells, more than the fixed scratch holds (" + std::to_string(kMaxShells) + ")");
    return PSC_EINVAL;
  }
  if (nshell_cap < nshell) {
    psc::set_error("psc_shell_spectra_noalloc: output arrays hold " + std::to_string(nshell_cap) +
                   " shells, " + std::to_string(nshell) + " needed");
    return PSC_EINVAL;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    psc::set_error(std::string("psc_shell_spectra_noalloc: no usable current device: ") + cudaGetErrorString(e));
    return PSC_ECUDA;
  }
  double* scratch = nullptr;
  {
    // once per device, with that device current: the host-side name of the
    // array is not a device address, so ask the runtime for the real one
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_ptr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_shell_scratch);
      if (e != cudaSuccess || !p) {
        psc::set_error(std::string("psc_shell_spectra_noalloc: cudaGetSymbolAddress failed: ") +
                       cudaGetErrorString(e));
        return PSC_ECUDA;
      }
      g_scratch_ptr[dev] = static_cast<double*>(p);
    }
    scratch = g_scratch_ptr[dev];
  }
  const psc::Dims d = psc::make_dims(N);
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  // every shell entry the finish kernel reads is rewritten by k_shells first,
  // so nothing left from an earlier call is read
  if (precision == PSC_FP64) {
    const unsigned char* u = static_cast<const unsigned char*>(state);
    psc::k_shells<double><<<nshell, 256, 0, st>>>(d, u, u + 3 * d.S * 16, nshell, scratch);
  } else {
    const unsigned char* u = static_cast<const unsigned char*>(state);
    psc::k_shells<float><<<nshell, 256, 0, st>>>(d, u, u + 3 * d.S * 8, nshell, scratch);
  }
  const double n3 = (double)N * N * N;
  k_noalloc_finish<<<(nshell + 127) / 128, 128, 0, st>>>(scratch, nshell, 1.0 / (2.0 * n3 * n3), Ek, Ephi);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    psc::set_error(std::string("psc_shell_spectra_noalloc: launch failed: ") + cudaGetErrorString(e));
    return PSC_ECUDA;
  }
  return PSC_OK;
}
