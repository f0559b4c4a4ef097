// The FMM product without any device allocation (xrl_fmm_mvm_device_noalloc).
//
// Some callers cannot allocate GPU memory at the moment they need a product:
// a latency-critical loop where a cudaMalloc could stall or fail, or a host
// framework whose own allocator owns the device memory budget and forbids
// allocations behind its back.  For them the working buffers
// of one product live in a fixed, statically declared device array; the
// setup products of the context (near field, moments, operators, tree) were
// allocated once by xrl_setup and are only read here.
#include <mutex>
#include <new>

#include "xrl_internal.hpp"

namespace {

constexpr size_t kScratchBytes = XRL_NOALLOC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Host code must not use g_noalloc_scratch directly (it names a host-side
// shadow, not device memory): the device address is looked up once per device.
constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

void* scratch_address(int device) {
  XRL_CHECK(device >= 0 && device < kMaxDevices, XRL_EINVAL, "device ordinal out of range for the scratch table");
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_addr[device]) {
    int cur = -1;
    XRL_CUDA(cudaGetDevice(&cur));
    XRL_CHECK(cur == device, XRL_ESTATE, "internal: scratch lookup with the wrong device current");
    void* p = nullptr;
    XRL_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    XRL_CHECK(p != nullptr, XRL_ECUDA, "cudaGetSymbolAddress returned no address");
    g_scratch_addr[device] = p;
  }
  return g_scratch_addr[device];
}

// Restores the caller's current device on every exit path.
struct DeviceGuard {
  int prev = -1;
  DeviceGuard() {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

}  // namespace

extern "C" xrl_status xrl_fmm_mvm_device_noalloc(xrl_ctx* c, int32_t nc, const double* dx, double* dy,
                                                 void* stream) {
  if (!c) return XRL_EINVAL;
  try {
    XRL_CHECK(c->ready, XRL_ESTATE, "call xrl_setup first");
    XRL_CHECK(nc > 0 && dx && dy, XRL_EINVAL, "bad mvm arguments");
    const size_t n = (size_t)c->N * nc;
    const size_t ne = (size_t)c->tree.n_boxes() * c->ncoef * nc;
    // four 256-byte aligned regions: X, Y, M, L
    auto up = [](size_t bytes) { return (bytes + 255) & ~(size_t)255; };
    const size_t need = 2 * up(n * sizeof(double)) + 2 * up(ne * sizeof(double));
    if (need > kScratchBytes) {
      c->err = "xrl_fmm_mvm_device_noalloc: needs " + std::to_string(need) + " bytes of scratch for " +
               std::to_string(nc) + " columns, more than the fixed " + std::to_string(kScratchBytes) +
               "-byte array; use fewer columns or xrl_fmm_mvm_device";
      return XRL_EINVAL;
    }
    DeviceGuard dg;
    XRL_CUDA(cudaSetDevice(c->device));
    unsigned char* base = static_cast<unsigned char*>(scratch_address(c->device));
    double* X = reinterpret_cast<double*>(base);
    double* Y = reinterpret_cast<double*>(base + up(n * sizeof(double)));
    double* Mx = reinterpret_cast<double*>(base + 2 * up(n * sizeof(double)));
    double* Lx = reinterpret_cast<double*>(base + 2 * up(n * sizeof(double)) + up(ne * sizeof(double)));
    cudaStream_t s = stream ? (cudaStream_t)stream : c->stream;
    // The plain FP64 kernels read only setup products.  Two switches of the
    // context would reach lazily allocated buffers or event objects: the
    // profiler (events) and the FP64-accurate residual mode of mixed solves
    // (double-float and integer-slice images); both are held off for the call.
    const bool prof = c->prof.on, df64 = c->df64_m2l;
    c->prof.on = false;
    c->df64_m2l = false;
    struct Restore {
      xrl_ctx* c;
      bool prof, df64;
      ~Restore() {
        c->prof.on = prof;
        c->df64_m2l = df64;
      }
    } restore{c, prof, df64};
    const int64_t peak0 = c->alloc.peak, cur0 = c->alloc.cur;
    xrl::launch_to_morton(c, nc, dx, X, s);
    xrl::fmm_apply_into(c, nc, X, Y, Mx, Lx, s);
    xrl::launch_from_morton(c, nc, Y, dy, s);
    XRL_CUDA(cudaGetLastError());
    XRL_CHECK(c->alloc.cur == cur0 && c->alloc.peak == peak0, XRL_ESTATE,
              "internal: the allocation-free product allocated device memory");
    c->err.clear();
    return XRL_OK;
  } catch (const xrl::Error& e) {
    c->err = e.what();
    return e.code;
  } catch (const std::bad_alloc&) {
    c->err = "host allocation failed";
    return XRL_ENOMEM;
  } catch (const std::exception& e) {
    c->err = e.what();
    return XRL_EINVAL;
  } catch (...) {
    c->err = "unknown error";
    return XRL_EINVAL;
  }
}
