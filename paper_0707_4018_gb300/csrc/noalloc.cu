// A fine-level MR smoother that allocates nothing (mg_smooth_fine_noalloc).
//
// Some callers cannot allocate device memory at the point where they smooth:
// code running while a CUDA stream is being captured into a graph (cudaMalloc
// is not permitted there), code inside a framework that owns the whole memory
// pool and forbids outside allocations, or latency-critical loops that must not
// pay for an allocation. For them this entry point keeps its scratch (the MR
// residual, A r, and the reduction partials / ticket / scalars) in one
// file-scope device array of fixed size, so a call needs only its inputs and
// outputs.
//
// Limits and sharing: the array holds a lattice of at most 65536 sites
// (256 x 256) and occupies about 4 MB on every GPU that loads this library,
// until the process exits. Every call on a device uses the same array and
// leaves its contents behind; the reduction ticket, which must start at zero,
// is cleared at the start of every call. Calls whose work overlaps on the GPU
// (different streams, or different host threads) race on the array.
#include <mutex>

#include "kernels.h"

namespace mg {

constexpr long long kNoAllocMaxSites = 65536;            // 256 x 256
constexpr long long kNoAllocMaxDofs = 2 * kNoAllocMaxSites;  // two spin components
constexpr int kNoAllocMaxBlocks = 512;                   // reduction blocks for n <= kNoAllocMaxDofs
// layout in doubles: r (2 n), Ar (2 n), partials (3 * blocks), scalars (8), ticket (8)
constexpr long long kNoAllocDoubles = 4 * kNoAllocMaxDofs + 3 * kNoAllocMaxBlocks + 8 + 8;

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

// Host code cannot use g_noalloc_scratch as a device address: the name is a
// host-side stand-in. The device address is looked up once per device, with
// that device current, on the first call there.
static std::mutex g_noalloc_mutex;
static void *g_noalloc_ptr[128] = {};

static double *noalloc_scratch() {
  int dev = 0;
  MG_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 128) fail(MG_ERR_UNSUPPORTED, "device ordinal beyond 127");
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (g_noalloc_ptr[dev] == nullptr) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr)
      fail(MG_ERR_CUDA, std::string("cudaGetSymbolAddress of the smoother scratch: ") + cudaGetErrorString(e));
    g_noalloc_ptr[dev] = p;
  }
  return static_cast<double *>(g_noalloc_ptr[dev]);
}

}  // namespace mg

using namespace mg;

extern "C" int mg_smooth_fine_noalloc(const mg_geom *g, const void *U, double m, const void *b, void *x, int nu,
                                      double omega, void *stream) {
  try {
    if (!g) fail(MG_ERR_INVALID_ARG, "null geometry");
    if (g->d != 2 || g->Nc != 1) fail(MG_ERR_UNSUPPORTED, "only d = 2, Nc = 1 is built");
    if (g->dims[0] < 2 || g->dims[1] < 2) fail(MG_ERR_INVALID_ARG, "lattice extents must be >= 2");
    const long long sites = (long long)g->dims[0] * g->dims[1];
    if (sites > kNoAllocMaxSites)
      fail(MG_ERR_INVALID_ARG, "lattice of " + std::to_string(sites) +
                                   " sites exceeds the no-allocation smoother's limit of 65536 sites (256 x 256)");
    if (!U || !b || !x) fail(MG_ERR_INVALID_ARG, "null pointer");
    if (b == x) fail(MG_ERR_INVALID_ARG, "b and x must not alias");
    if (nu < 0) fail(MG_ERR_INVALID_ARG, "nu must be >= 0");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const long long n = 2 * sites;
    // the scratch address belongs to the current device: x must live there too
    int dev = 0;
    MG_CUDA(cudaGetDevice(&dev));
    cudaPointerAttributes pa{};
    if (cudaPointerGetAttributes(&pa, x) != cudaSuccess || pa.type != cudaMemoryTypeDevice || pa.device != dev) {
      (void)cudaGetLastError();
      fail(MG_ERR_INVALID_ARG, "x must be device memory of the current device (the scratch array is per device)");
    }
    double *S = noalloc_scratch();
    Cx<double> *r = reinterpret_cast<Cx<double> *>(S);
    Cx<double> *Ar = r + kNoAllocMaxDofs;
    double *partials = S + 4 * kNoAllocMaxDofs;
    double *sc = partials + 3 * kNoAllocMaxBlocks;
    unsigned int *ticket = reinterpret_cast<unsigned int *>(sc + 8);
    ReduceWs ws{partials, ticket, kNoAllocMaxBlocks, 3LL * kNoAllocMaxBlocks};
    const Geo2 geo{g->dims[0], g->dims[1], sites};
    const Cx<double> *Ud = static_cast<const Cx<double> *>(U);
    Cx<double> *xd = static_cast<Cx<double> *>(x);
    MG_CUDA(cudaMemsetAsync(ticket, 0, sizeof(unsigned int), s));
    launch_zero<double>(xd, n, s);
    launch_copy<double>(static_cast<const Cx<double> *>(b), r, n, s);
    for (int i = 0; i < nu; ++i) {
      launch_dslash<double>(Ud, r, Ar, geo, g->d + m, nullptr, 1.0, 0.0, s);
      launch_dot_norm<double>(Ar, r, n, sc, ws, s);
      launch_mr_update<double>(sc, omega, xd, r, Ar, n, s);
    }
    set_last_error("");
    return MG_OK;
  } catch (const Error &e) {
    set_last_error(e.msg);
    return e.code;
  } catch (...) {
    set_last_error("unexpected exception");
    return MG_ERR_CUDA;
  }
}
