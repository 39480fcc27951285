// tdc_noalloc.cu -- tdc_eig_noalloc: the eigensolver for callers that cannot
// allocate device memory.
//
// Some callers cannot call cudaMalloc: code that runs inside a process whose
// device memory is already fully reserved by another allocator (a framework's
// caching pool, a pre-sized arena), plugins that are not allowed to touch the
// allocator, and latency-critical callers for which an allocation that may
// block or fail is not acceptable.  They still own their inputs and outputs but
// cannot provide the workspace tdc_eig needs.  For them this entry point runs
// the same solver with its workspace in a fixed-size array that lives in the
// library's own device memory: a file-scope __device__ array that every GPU
// which loads the library holds until the process exits.
//
// The array's name is only a host-side stand-in in host code, so its device
// address is looked up once per device (with that device current) through
// cudaGetSymbolAddress on the first call made on that device; that first call
// should therefore come before any stream capture.  Every call shares the one
// array: calls that overlap on the GPU (two streams, two threads) race on it
// and must be ordered by the caller.  The array keeps the previous call's
// contents; the solver writes every workspace entry before it reads it, so
// nothing has to be cleared between calls.  No cudaMalloc, cudaFree or other
// allocating routine is called on this path; statistics collection (which
// would create CUDA events) is switched off here.
#include <mutex>

#include "tdc_common.cuh"

namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)24 << 20;  // 24 MiB
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_noalloc_mu;
void* g_noalloc_addr[64];

// Device address of the scratch array on the current device (NULL on failure).
void* noalloc_scratch() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress((void**)&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) return nullptr;
    g_noalloc_addr[dev] = p;
  }
  return g_noalloc_addr[dev];
}

}  // namespace

extern "C" int tdc_eig_noalloc(int64_t n, const double* d, const double* e, double* lam, double* Q, int64_t ldq,
                               const tdc_opts* o, tdc_stream_t stream) {
  tdc_opts op;
  tdc_default_opts(&op);
  if (o) op = *o;
  op.collect_stats = 0;
  if (n < 0) return -1;
  if (n == 0) return TDC_OK;
  size_t need = 0;
  int ws_status = tdc_workspace_size(n, &op, &need);
  if (ws_status != TDC_OK) return ws_status == -1 ? -1 : -7;
  if (need > kNoAllocScratchBytes && op.merge_mode == TDC_MERGE_AUTO) {
    // the library's choice: without room for the split path's digit images, the FP64 merge
    op.merge_mode = TDC_MERGE_DENSE;
    ws_status = tdc_workspace_size(n, &op, &need);
    if (ws_status != TDC_OK) return -7;
  }
  if (need > kNoAllocScratchBytes) return TDC_ETOOLARGE;
  void* ws = noalloc_scratch();
  if (!ws) return TDC_ECUDA;
  return tdc_eig(n, d, e, lam, Q, ldq, ws, kNoAllocScratchBytes, &op, stream);
}
