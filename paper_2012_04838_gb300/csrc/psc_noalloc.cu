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

// Whether p is device memory (or managed memory) that device `dev` owns;
// otherwise `why` says what it is.
bool on_device(const void* p, int dev, const char* name, std::string& why) {
  cudaPointerAttributes at;
  const cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) {
    cudaGetLastError();  // the failed query leaves a (non-sticky) error: clear it
    why = std::string(name) + ": not a pointer CUDA knows (" + cudaGetErrorString(e) + ")";
    return false;
  }
  if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) {
    why = std::string(name) + (at.type == cudaMemoryTypeHost ? " is pinned host memory"
                                                            : " is host memory unknown to CUDA") +
          ", not device memory";
    return false;
  }
  if (at.type == cudaMemoryTypeDevice && at.device != dev) {
    why = std::string(name) + " lives on device " + std::to_string(at.device) + ", not on the current device " +
          std::to_string(dev);
    return false;
  }
  return true;
}

}  // namespace

namespace psc {
void set_error(const std::string& msg);
}

extern "C" psc_status psc_shell_spectra_noalloc(const void* state, int32_t N, int32_t precision,
                                                int32_t dealias, double* Ek, double* Ephi, int32_t nshell_cap,
                                                void* stream) {
  // argument checks that need no GPU come first
  if (!state || !Ek || !Ephi) {
    psc::set_error("psc_shell_spectra_noalloc: null pointer");
    return PSC_EINVAL;
  }
  if (N < 8 || N > 65536 || (precision != PSC_FP64 && precision != PSC_FP32_MIXED) ||
      (dealias != PSC_DEALIAS_TWO_THIRDS && dealias != PSC_DEALIAS_PHASE_SHIFT)) {
    psc::set_error("psc_shell_spectra_noalloc: N must be 8..65536, precision PSC_FP64 or PSC_FP32_MIXED, "
                   "dealias PSC_DEALIAS_TWO_THIRDS or PSC_DEALIAS_PHASE_SHIFT");
    return PSC_EINVAL;
  }
  // the same layout and shell count as a simulation with these parameters
  const psc::Dims d = psc::make_dims(N, dealias == PSC_DEALIAS_PHASE_SHIFT);
  const int nshell = psc::shell_count(d);
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
  if (e != cudaSuccess) {
    psc::set_error(std::string("psc_shell_spectra_noalloc: no usable current device: ") + cudaGetErrorString(e));
    return PSC_ECUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    psc::set_error("psc_shell_spectra_noalloc: current device " + std::to_string(dev) + " is beyond the " +
                   std::to_string(kMaxDevices) + " devices this call keeps scratch addresses for");
    return PSC_EINVAL;
  }
  // a pointer the kernels cannot read on this device is an argument error,
  // reported before anything is launched
  std::string why;
  if (!on_device(state, dev, "state", why) || !on_device(Ek, dev, "Ek", why) || !on_device(Ephi, dev, "Ephi", why)) {
    psc::set_error("psc_shell_spectra_noalloc: " + why);
    return PSC_EINVAL;
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
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  // every shell entry the finish kernel reads is rewritten by k_shells first,
  // so nothing left from an earlier call is read
  const unsigned char* u = static_cast<const unsigned char*>(state);
  if (precision == PSC_FP64)
    psc::k_shells<double><<<nshell, 256, 0, st>>>(d, u, u + 3 * d.S * 16, nshell, scratch);
  else
    psc::k_shells<float><<<nshell, 256, 0, st>>>(d, u, u + 3 * d.S * 8, nshell, scratch);
  const double n3 = (double)N * N * N;
  k_noalloc_finish<<<(nshell + 127) / 128, 128, 0, st>>>(scratch, nshell, 1.0 / (2.0 * n3 * n3), Ek, Ephi);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    psc::set_error(std::string("psc_shell_spectra_noalloc: launch failed: ") + cudaGetErrorString(e));
    return PSC_ECUDA;
  }
  return PSC_OK;
}
