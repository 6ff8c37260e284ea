// Allocation-free transmission entry point.
//
// Some callers cannot allocate device memory at all: code running inside a
// memory pool that owns the whole device, a host process that must not grow
// its footprint after start-up, or a framework hook that is forbidden from
// calling cudaMalloc / cudaMallocAsync while its own allocator is active.
// For them this file provides ss_caroli_transmission_noalloc, which computes
// the same T[p] = Re Tr[Gamma_L G_1n Gamma_R G_1n^H] as
// ss_caroli_transmission but takes every byte of scratch (the Gamma blocks,
// the two products, the traces and the launch descriptors) from one
// file-scope device array of fixed size.  Every GPU that loads the library
// holds that array until the process exits.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "splitsolve.h"
#include "ss_internal.cuh"

using namespace ss;

namespace {

// Limits of the static scratch: n_pts * s_b^2 <= 65536 complex per block kind
// (e.g. one point of s_b = 256, or 64 points of s_b = 32), n_pts <= 256.
constexpr size_t NA_MAX_ELEMS = 65536;
constexpr int NA_MAX_POINTS = 256;
constexpr size_t NA_DATA_BYTES = (4 * NA_MAX_ELEMS + NA_MAX_POINTS) * sizeof(z64);
constexpr size_t NA_DESC_BYTES =
    NA_MAX_POINTS * (2 * sizeof(FormDesc) + 2 * sizeof(GemmDesc) + sizeof(TraceDesc) + 4 * sizeof(int)) + 1024;
constexpr size_t NA_TOTAL_BYTES = NA_DATA_BYTES + NA_DESC_BYTES;

// The scratch itself.  In host code this name is only a stand-in for the
// symbol; its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_na_scratch[NA_TOTAL_BYTES];

constexpr int NA_MAX_DEVICES = 64;
std::mutex g_na_mutex;
void* g_na_addr[NA_MAX_DEVICES] = {nullptr};
// The error text belongs to the calling thread, so callers on different
// threads (e.g. one per device) never overwrite each other's message.
thread_local std::string g_na_error;

// Device address of the scratch on the current device, looked up once per
// device (the first call on a device does this set-up).
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= NA_MAX_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_na_mutex);
  if (!g_na_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_na_scratch);
    if (e != cudaSuccess) return e;
    g_na_addr[dev] = p;
  }
  *out = g_na_addr[dev];
  return cudaSuccess;
}

size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

template <class D>
size_t append(std::vector<unsigned char>& buf, const std::vector<D>& v) {
  const size_t off = align16(buf.size());
  buf.resize(off + v.size() * sizeof(D));
  if (!v.empty()) std::memcpy(buf.data() + off, v.data(), v.size() * sizeof(D));
  return off;
}

int na_fail(int code, const std::string& msg) {
  g_na_error = msg;
  return code;
}

}  // namespace

extern "C" const char* ss_noalloc_last_error(void) { return g_na_error.c_str(); }

extern "C" int ss_caroli_transmission_noalloc(int n_pts, int s_b, const ss_c64* sigma_L, const ss_c64* sigma_R,
                                              const ss_c64* G1n, double* T, void* stream) {
  g_na_error.clear();
  if (n_pts < 0 || s_b < 1) return na_fail(SS_ERR_ARG, "bad sizes");
  if (n_pts == 0) return SS_OK;
  if (!sigma_L || !sigma_R || !G1n || !T) return na_fail(SS_ERR_ARG, "NULL array");
  if (n_pts > NA_MAX_POINTS || (size_t)n_pts * s_b * s_b > NA_MAX_ELEMS)
    return na_fail(SS_ERR_ARG, "problem exceeds the static scratch: need n_pts <= 256 and n_pts*s_b^2 <= 65536, got n_pts=" +
                                   std::to_string(n_pts) + " s_b=" + std::to_string(s_b));
  cudaStream_t st = (cudaStream_t)stream;
  // The call synchronises its stream and copies its descriptors from a
  // temporary host buffer, so it cannot be recorded into a CUDA graph.
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(st, &cap);
  if (e != cudaSuccess) return na_fail(SS_ERR_CUDA, std::string("cudaStreamIsCapturing: ") + cudaGetErrorString(e));
  if (cap != cudaStreamCaptureStatusNone) return na_fail(SS_ERR_ARG, "the stream is being captured; this call cannot be captured");
  void* base = nullptr;
  e = scratch_address(&base);
  if (e != cudaSuccess) return na_fail(SS_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
  unsigned char* dbase = static_cast<unsigned char*>(base);
  z64* data = reinterpret_cast<z64*>(dbase);
  unsigned char* desc = dbase + NA_DATA_BYTES;

  // Every scratch byte that is read is written earlier in this call, so
  // nothing needs clearing between calls.
  std::vector<FormDesc> f;
  std::vector<GemmDesc> g;
  std::vector<TraceDesc> t;
  caroli_descriptors(n_pts, s_b, reinterpret_cast<const z64*>(sigma_L), reinterpret_cast<const z64*>(sigma_R),
                     reinterpret_cast<const z64*>(G1n), data, f, g, t);
  std::vector<int> fstart(f.size()), gstart(g.size());
  int ftot = 0, gtot = 0;
  for (size_t i = 0; i < f.size(); ++i) { fstart[i] = ftot; ftot += zform_tiles(f[i].rows, f[i].cols); }
  for (size_t i = 0; i < g.size(); ++i) { gstart[i] = gtot; gtot += zgemm_tiles(g[i].m, g[i].n); }
  std::vector<unsigned char> host;
  const size_t of = append(host, f), ofs = append(host, fstart);
  const size_t og = append(host, g), ogs = append(host, gstart);
  const size_t ot = append(host, t);
  if (host.size() > NA_DESC_BYTES) return na_fail(SS_ERR_ARG, "descriptor area too small");
  e = cudaMemcpyAsync(desc, host.data(), host.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    launch_zform(reinterpret_cast<const FormDesc*>(desc + of), reinterpret_cast<const int*>(desc + ofs),
                 (int)f.size(), ftot, st);
    launch_zgemm(reinterpret_cast<const GemmDesc*>(desc + og), reinterpret_cast<const int*>(desc + ogs),
                 (int)g.size(), gtot, st);
    launch_trace(reinterpret_cast<const TraceDesc*>(desc + ot), (int)t.size(), st);
    launch_real_part(data + (size_t)n_pts * 4 * s_b * s_b, T, n_pts, st);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return na_fail(SS_ERR_CUDA, cudaGetErrorString(e));
  return SS_OK;
}
