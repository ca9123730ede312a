// mt_static.cu -- mt_certify_static: the root certificate without any
// caller-provided workspace and without any device allocation.
//
// Who needs it: code that runs where cudaMalloc is not an option -- inside
// a host callback or an allocator hook, in a process whose memory is fully
// reserved by another runtime's pool, or in a plug-in that must not touch
// the host application's allocator.  Such callers pass only their input
// roots and their output arrays.
//
// The scratch (sort keys, permutation, radix histograms and the counters)
// lives in one file-scope __device__ array of MT_CERTIFY_STATIC_BYTES.
// Every GPU that loads this library holds that array until the process
// exits.  In host code the array's name is only a host-side stand-in, so
// the device address is looked up once per device with
// cudaGetSymbolAddress(), the device being current, on the first call of
// mt_certify_static on that device; that first call should therefore come
// before any stream capture.  Every call shares the array: calls that
// overlap on the GPU (different streams, or different host threads without
// ordering) race on it.  The counters are re-initialised by each call; the
// rest of the array is fully rewritten before it is read.
#include <cstdio>
#include <cstring>
#include <mutex>

#include "../../include/mtsplit.h"
#include "mt_internal.h"

namespace {

using namespace mt;

constexpr size_t kStaticBytes = (size_t)MT_CERTIFY_STATIC_BYTES;

__device__ __align__(256) unsigned char g_certify_scratch[kStaticBytes];

std::mutex g_mu;
void* g_addr[64] = {nullptr};

mt_status static_fail(mt_status st, const char* msg, cudaError_t e = cudaSuccess) {
  char buf[256];
  if (e != cudaSuccess)
    snprintf(buf, sizeof(buf), "mt_certify_static: %s: %s", msg, cudaGetErrorString(e));
  else
    snprintf(buf, sizeof(buf), "mt_certify_static: %s", msg);
  set_error_message(buf);  // reported by mt_last_error()
  return st;
}

size_t al(size_t x) { return (x + 255) & ~size_t(255); }

// Device address of the scratch array on the current device (looked up once).
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_certify_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" MT_API mt_status mt_certify_static(int kind, int l, int n, const double* d_roots,
                                              int64_t count, double tol, uint8_t* d_pass,
                                              double* d_radius, int64_t* n_pass, void* stream) {
  set_error_message("");
  if (kind == 2) return static_fail(MT_EINVAL, "q_{l,n} (kind 2) is certified by mt_certify only");
  if (!valid_poly(kind, kind == 0 ? 0 : l, n)) return static_fail(MT_EINVAL, "polynomial out of range");
  if (count < 0 || (count > 0 && (!d_roots || !d_pass))) return static_fail(MT_EINVAL, "bad buffers");
  if (count > MT_CERTIFY_STATIC_MAX_ROOTS)
    return static_fail(MT_ECAPACITY, "mt_certify_static takes at most MT_CERTIFY_STATIC_MAX_ROOTS roots");
  // carve the static array: counters, keys, keys_alt, vals, vals_alt, radix temp
  const int64_t c = count > 0 ? count : 1;
  const size_t o_keys = al(sizeof(DevCounters));
  const size_t o_keys2 = o_keys + al((size_t)c * 8);
  const size_t o_vals = o_keys2 + al((size_t)c * 8);
  const size_t o_vals2 = o_vals + al((size_t)c * 4);
  const size_t o_rtmp = o_vals2 + al((size_t)c * 4);
  const size_t need = o_rtmp + al(radix_temp_bytes(c));
  if (need > kStaticBytes) return static_fail(MT_ENOMEM, "static scratch too small");
  void* base = nullptr;
  cudaError_t e = scratch_address(&base);
  if (e != cudaSuccess) return static_fail(MT_ECUDA, "cudaGetSymbolAddress failed", e);
  char* b = (char*)base;
  DevCounters* ctr = (DevCounters*)b;
  uint64_t* keys = (uint64_t*)(b + o_keys);
  uint64_t* keys2 = (uint64_t*)(b + o_keys2);
  uint32_t* vals = (uint32_t*)(b + o_vals);
  uint32_t* vals2 = (uint32_t*)(b + o_vals2);
  void* rtmp = (void*)(b + o_rtmp);
  cudaStream_t s = (cudaStream_t)stream;
  const PolyDev P = make_poly(kind, kind == 0 ? 0 : l, n);
  if (tol <= 0) tol = 1e-12;
  if ((e = launch_init_counters(ctr, s)) != cudaSuccess) return static_fail(MT_ECUDA, "launch", e);
  if ((e = launch_keys_plain((const double2*)d_roots, count, keys, vals, s)) != cudaSuccess)
    return static_fail(MT_ECUDA, "launch", e);
  if ((e = radix_sort_pairs(keys, vals, keys2, vals2, count, rtmp, s)) != cudaSuccess)
    return static_fail(MT_ECUDA, "launch", e);
  if ((e = launch_certify_list(P, (const double2*)d_roots, vals, count, tol, d_pass, d_radius, ctr,
                               s)) != cudaSuccess)
    return static_fail(MT_ECUDA, "launch", e);
  unsigned long long h = 0;
  if ((e = cudaMemcpyAsync(&h, &ctr->n_cert_pass, sizeof(h), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return static_fail(MT_ECUDA, "cudaMemcpyAsync", e);
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return static_fail(MT_ECUDA, "sync", e);
  if (n_pass) *n_pass = (int64_t)h;
  return MT_OK;
}
