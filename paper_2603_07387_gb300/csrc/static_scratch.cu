// static_scratch.cu -- tnsk_estimate_static: the method-1 estimate for callers
// that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: plugins whose host application owns every
// allocation (a fixed memory pool or an allocator that forbids side
// allocations), or embedded uses that must not grow device memory after
// start-up. For them this entry point runs the same kernels as tnsk_estimate
// with TNSK_GENERAL, but keeps every piece of scratch (launch descriptors, hash
// tables, sketches, per-rep estimates, FFT twiddles) in one file-scope device
// array of fixed size. It allocates nothing: no cudaMalloc, no cudaFree, no
// allocating library call.
//
// Costs and rules:
//  - The array (kStaticBytes = 16 MiB) is part of the library's device image:
//    every GPU that loads libtnsk holds it until the process exits.
//  - All calls share the array, which keeps the last call's contents. Calls on
//    different devices are independent (each device has its own copy of the
//    array). Calls on one device whose GPU work overlaps, from two streams or two
//    host threads, race on the array: order them on one stream.
//  - The first call on a device looks up the array's device address
//    (cudaGetSymbolAddress) and writes the twiddle tables with a synchronous
//    copy.
//  - Hyperedges (a mode in several contractions) get WLOG 1's copy tensors as in
//    tnsk_estimate; the copy tensors are never stored, so this needs no buffer.
#include <cmath>
#include <mutex>
#include <vector>

#include "kernels.cuh"
#include "method2.cuh"
#include "normalize.cuh"
#include "plan.cuh"

namespace tnsk {
namespace {

constexpr size_t kStaticBytes = (size_t)16 << 20;
constexpr int kMaxDevices = 64;
constexpr int kLog2Levels = 17;  // twiddle tables for m = 2^0 .. 2^16

static __device__ __align__(256) unsigned char g_tnsk_static_scratch[kStaticBytes];

struct StaticDevice {
    bool ready = false;
    unsigned char* base = nullptr;  // device address of g_tnsk_static_scratch
    size_t arena_off = 0;           // first byte free for per-call scratch
    size_t tw_ptrs_off = 0;         // device array of the FP32 twiddle pointers
};

std::mutex g_setup_mutex;
StaticDevice g_devices[kMaxDevices];

// Once per device, with that device current: find the array and fill the FP32
// twiddle tables tw[k] = exp(-2 pi i k/m), k < m/2 (host FP64, rounded to FP32).
tnsk_status setup_device(int dev, StaticDevice*& out) {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    StaticDevice& sd = g_devices[dev];
    if (!sd.ready) {
        void* ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_tnsk_static_scratch) != cudaSuccess || !ptr) {
            cudaGetLastError();
            return TNSK_ERR_CUDA;
        }
        unsigned char* base = (unsigned char*)ptr;
        std::vector<float> tw;
        std::vector<size_t> off;
        for (int l = 0; l < kLog2Levels; ++l) {
            size_t m = (size_t)1 << l, M = l > 0 ? m / 2 : 1;
            off.push_back(tw.size() * sizeof(float));
            for (size_t k = 0; k < M; ++k) {
                double a = -2.0 * M_PI * (double)k / (double)m;
                tw.push_back((float)std::cos(a));
                tw.push_back((float)std::sin(a));
            }
        }
        size_t tw_bytes = tw.size() * sizeof(float);
        size_t ptrs_off = (tw_bytes + 255) & ~(size_t)255;
        std::vector<const void*> ptrs;
        for (int l = 0; l < kLog2Levels; ++l) ptrs.push_back(base + off[l]);
        if (cudaMemcpy(base, tw.data(), tw_bytes, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(base + ptrs_off, ptrs.data(), ptrs.size() * sizeof(void*), cudaMemcpyHostToDevice) !=
                cudaSuccess) {
            cudaGetLastError();
            return TNSK_ERR_CUDA;
        }
        sd.base = base;
        sd.tw_ptrs_off = ptrs_off;
        sd.arena_off = (ptrs_off + ptrs.size() * sizeof(void*) + 255) & ~(size_t)255;
        sd.ready = true;
    }
    out = &sd;
    return TNSK_OK;
}

}  // namespace
}  // namespace tnsk

using namespace tnsk;

extern "C" tnsk_status tnsk_estimate_static(const tnsk_network* net, const tnsk_params* params, double* out,
                                            double* per_rep, void* cuda_stream) {
    if (!net || !params || !out) return TNSK_ERR_INVALID;
    if (params->method != TNSK_GENERAL || params->prec != TNSK_PREC_FP32) return TNSK_ERR_UNSUPPORTED;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return TNSK_ERR_CUDA;
    }
    // WLOG 1 (Sec. 4.1) for hyperedges: a host-side view of the network with copy
    // tensors appended; method-1 networks never need a rewritten tensor buffer
    NormBatch nb;
    std::string why;
    tnsk_status st = normalize_batch(1, net, params, nb, why);
    if (st != TNSK_OK) return st;
    if (!nb.jobs.empty()) return TNSK_ERR_UNSUPPORTED;
    const tnsk_network* view = nb.used ? nb.view.data() : net;
    const char* diag = !nb.diag.empty() && !nb.diag[0].empty() ? nb.diag[0].data() : nullptr;
    std::vector<NetInfo> infos(1);
    st = validate(*view, *params, infos[0], why, false, diag);
    if (st != TNSK_OK) return st;
    StaticDevice* sd = nullptr;
    st = setup_device(dev, sd);
    if (st != TNSK_OK) return st;
    BatchPlan plan;
    plan.arena.used = sd->arena_off;  // per-call regions start after the twiddles
    double* outs[1] = {out};
    double* pers[1] = {per_rep};
    st = plan_batch(infos, view, params, outs, pers, false, false, plan, why);
    if (st != TNSK_OK) return st;
    if (plan.arena.used > kStaticBytes) return TNSK_ERR_UNSUPPORTED;  // beyond the fixed 16 MiB
    cudaStream_t s = (cudaStream_t)cuda_stream;
    unsigned char* base = sd->base;
    const void* const* tws = (const void* const*)(base + sd->tw_ptrs_off);
    if (!plan.host_desc.empty() &&
        cudaMemcpyAsync(base + plan.desc_off, plan.host_desc.data(), plan.host_desc.size(), cudaMemcpyHostToDevice,
                        s) != cudaSuccess)
        return TNSK_ERR_CUDA;
    // sketches and per-rep estimates accumulate: they must start at zero
    if (plan.zero_bytes && cudaMemsetAsync(base + plan.zero_off, 0, plan.zero_bytes, s) != cudaSuccess)
        return TNSK_ERR_CUDA;
    if (launch_draw_tables((const TabReq*)(base + plan.reqs_off), plan.n_reqs, plan.n_table_rows,
                           (uint32_t*)(base + plan.tabs_off), s) != cudaSuccess ||
        launch_m1_scatters(plan, base, base + plan.m1.xs_off, false, s) != cudaSuccess ||
        launch_m1_diag(plan, base, base + plan.m1.xs_off, false, s) != cudaSuccess ||
        launch_m1_spectra(plan, base, base + plan.m1.xs_off, (const void* const*)tws, false, s) != cudaSuccess ||
        launch_combine((const CombineItem*)(base + plan.comb_off), plan.n_comb, (const double*)(base + plan.yrep_off),
                       s) != cudaSuccess) {
        cudaGetLastError();
        return TNSK_ERR_CUDA;
    }
    return TNSK_OK;
}
