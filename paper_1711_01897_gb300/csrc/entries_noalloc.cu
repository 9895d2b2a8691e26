// bem_entries_noalloc: the dense sub-block request of bem_entries for
// callers that must not allocate device memory while they run.  The list of
// singular pairs that bem_entries keeps in stream-ordered scratch lives here
// in one file-scope device array instead.
#include <algorithm>
#include <map>
#include <mutex>
#include <new>
#include <string>

#include "../../include/bem.h"
#include "bem_internal.h"

namespace bem {
namespace {

// Capacity of the static scratch: singular pairs per case (vertex, edge,
// identical).  3 * 2^18 * 16 bytes = 12 MiB plus counters, held by every GPU
// that loads the library until the process exits.
constexpr int64_t kNoAllocPairs = int64_t(1) << 18;
constexpr size_t kListBytes = kNoAllocPairs * sizeof(SingPair);
constexpr size_t kScratchBytes = 3 * kListBytes + 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
std::map<int, unsigned char *> g_addr;  // device -> address of g_noalloc_scratch

// Device address of the scratch on the current device (host code may not use
// the symbol itself: in host code it names a host-side shadow).
cudaError_t scratch_address(int device, unsigned char **out)
{
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_addr.find(device);
    if (it != g_addr.end()) {
        *out = it->second;
        return cudaSuccess;
    }
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_addr[device] = static_cast<unsigned char *>(p);
    *out = static_cast<unsigned char *>(p);
    return cudaSuccess;
}

// True if p is device memory of `device` (or managed memory, which every
// device can reach).  Device memory of another GPU is refused: without peer
// access the kernels would fault on it.
bool on_device(const void *p, int device)
{
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == device;
}

int err(int code, const std::string &msg)
{
    set_last_error(msg.c_str());
    return code;
}

}  // namespace
}  // namespace bem

using namespace bem;

namespace {

int entries_noalloc(bem_mesh mesh, int32_t op, double k, int32_t prec, const int32_t *test_ids,
                    int64_t n_test, const int32_t *trial_ids, int64_t n_trial, void *out,
                    void *cuda_stream)
{
    set_last_error("");
    MeshView M;
    if (!mesh_view(mesh, &M)) return err(BEM_E_ARG, "null mesh");
    if (op < 0 || op > 2) return err(BEM_E_ARG, "bad op");
    if (prec != BEM_FP64 && prec != BEM_MIXED && prec != BEM_MIXED_SP) return err(BEM_E_ARG, "bad prec");
    if (!(k == k) || k - k != 0.0) return err(BEM_E_ARG, "bad k");
    if (n_test < 0 || n_trial < 0) return err(BEM_E_ARG, "negative size");
    if (n_test == 0 || n_trial == 0) return BEM_OK;
    if (!test_ids || !trial_ids || !out) return err(BEM_E_ARG, "null array");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != M.device)
        return err(BEM_E_STATE, "the mesh's device must be the current device");
    if (!on_device(test_ids, dev) || !on_device(trial_ids, dev) || !on_device(out, dev))
        return err(BEM_E_ARG, "bem_entries_noalloc takes device pointers on the mesh's device only");
    const int64_t need = std::min<int64_t>(n_test * n_trial,
                                           n_test * std::max<int64_t>(M.max_touch, 1));
    if (need > kNoAllocPairs)
        return err(BEM_E_ARG, "request may hold up to " + std::to_string(need) +
                                  " singular pairs per case; the allocation-free scratch holds " +
                                  std::to_string(kNoAllocPairs) + " (use bem_entries)");
    QuadRule rule;
    const SingTable *sing = nullptr;
    if (!consts_peek(dev, &rule, &sing))
        return err(BEM_E_STATE, "device constants missing (create the mesh on this device)");
    unsigned char *base = nullptr;
    cudaError_t e = scratch_address(dev, &base);
    if (e != cudaSuccess)
        return err(BEM_E_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    cudaStream_t st = (cudaStream_t)cuda_stream;
    SingPair *lists[3] = {(SingPair *)base, (SingPair *)(base + kListBytes),
                          (SingPair *)(base + 2 * kListBytes)};
    unsigned long long *counts = (unsigned long long *)(base + 3 * kListBytes);
    int *eflag = (int *)(counts + 3);
    int herr = 0;
    e = cudaMemsetAsync(counts, 0, 256, st);  // counters and error flag start at zero
    if (e == cudaSuccess)
        e = launch_entries_regular(M.g, rule, op, k, prec, test_ids, n_test, trial_ids, n_trial,
                                   out, lists, counts, (unsigned long long)kNoAllocPairs, eflag, st);
    const SingPair *cl[3] = {lists[0], lists[1], lists[2]};
    // the device counts, capped at the lists' capacity, say how many pairs
    // there are; the host bound `need` only sizes the grids
    int64_t hc[3] = {kNoAllocPairs, kNoAllocPairs, kNoAllocPairs};
    int64_t gc[3] = {need, need, need};
    if (e == cudaSuccess) e = launch_singular(M.g, sing, op, k, prec, cl, counts, hc, out, st, gc);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, eflag, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return err(BEM_E_CUDA, std::string("bem_entries_noalloc: ") + cudaGetErrorString(e));
    if (herr == 1) return err(BEM_E_ARG, "triangle id out of range");
    // repeated trial ids can make more touching pairs than the bound above
    // counts; the lists stopped at their capacity and `out` is undefined
    if (herr == 2)
        return err(BEM_E_ARG, "request holds more than " + std::to_string(kNoAllocPairs) +
                                  " singular pairs of one kind (repeated ids); the allocation-free "
                                  "scratch is full (use bem_entries)");
    return BEM_OK;
}

}  // namespace

extern "C" int bem_entries_noalloc(bem_mesh mesh, int32_t op, double k, int32_t prec,
                                   const int32_t *test_ids, int64_t n_test,
                                   const int32_t *trial_ids, int64_t n_trial, void *out,
                                   void *cuda_stream)
{
    // no exception may cross the C boundary (std::map and std::string can
    // throw on host allocation failure)
    try {
        return entries_noalloc(mesh, op, k, prec, test_ids, n_test, trial_ids, n_trial, out,
                               cuda_stream);
    } catch (const std::bad_alloc &) {
        return err(BEM_E_OOM, "host allocation failed");
    } catch (...) {
        return err(BEM_E_CUDA, "bem_entries_noalloc: unexpected exception");
    }
}
