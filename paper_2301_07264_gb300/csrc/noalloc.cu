// Allocation-free variant of arso_score_state.
//
// Some callers cannot call cudaMalloc: code that runs inside another
// allocator's arena (a framework that owns all device memory), code on a path
// where allocation is forbidden because it would synchronise the device or
// fail under memory pressure, or a host that must never grow its device
// footprint after start-up. arso_score_state_noalloc scores a state with the
// same kernels as arso_score_state, but its scratch (per-block criterion
// partials, the final score and the binning bitmap) lives in file-scope
// device arrays of fixed size instead of stream-ordered allocations.
//
// The arrays exist once per CUDA context that loads the library's module and
// stay allocated until the context ends (normally process exit). In host code
// the array names are host-side stand-ins, not device addresses, so every call
// looks up the device addresses with cudaGetSymbolAddress in the context
// current on the calling thread. The lookup allocates nothing; it is done per
// call rather than cached so that a device reset or a caller-made context never
// leaves a stale address behind. The first call in a context also loads the
// module there, so make it before any stream capture. All calls in a context
// share the arrays and the arrays keep the last call's contents: every call
// overwrites the bitmap words it uses and every partial it reads, and calls
// that overlap on the GPU race on them.
#include "kernels.h"

namespace arso {

constexpr uint32_t NOALLOC_MAX_BLOCKS = 152 * 8;          // criterion partials
constexpr uint32_t NOALLOC_MAX_BINNING_QUBITS = 20;       // bitmap of 2^20 bits = 128 KiB

static __device__ __align__(256) Partial g_noalloc_partials[NOALLOC_MAX_BLOCKS];
static __device__ __align__(256) double g_noalloc_score[1];
static __device__ __align__(256) uint32_t g_noalloc_bitmap[(1u << NOALLOC_MAX_BINNING_QUBITS) / 32];

namespace {
struct NoAllocPtrs {
    Partial *partials = nullptr;
    double *score = nullptr;
    uint32_t *bitmap = nullptr;
};

// device addresses of the file-scope arrays in the current context
NoAllocPtrs noalloc_setup() {
    void *a = nullptr, *b = nullptr, *c = nullptr;
    ARSO_CUDA(cudaGetSymbolAddress(&a, g_noalloc_partials));
    ARSO_CUDA(cudaGetSymbolAddress(&b, g_noalloc_score));
    ARSO_CUDA(cudaGetSymbolAddress(&c, g_noalloc_bitmap));
    NoAllocPtrs p;
    p.partials = static_cast<Partial *>(a);
    p.score = static_cast<double *>(b);
    p.bitmap = static_cast<uint32_t *>(c);
    return p;
}
}  // namespace

}  // namespace arso

using namespace arso;

extern "C" arso_status arso_score_state_noalloc(uint32_t n, const void *amps, const void *ref,
                                                const arso_criterion *crit, void *stream, double *score_out) {
    try {
        ARSO_REQUIRE(amps && crit && score_out, "NULL argument");
        ARSO_REQUIRE(n >= 1 && n <= 34, "n_qubits must be in [1, 34]");
        ARSO_REQUIRE(crit->kind <= ARSO_CRIT_ARGMAX, "bad criterion kind");
        ARSO_REQUIRE(crit->kind != ARSO_CRIT_FIDELITY || ref != nullptr, "fidelity needs ref");
        const uint64_t N = 1ull << n;
        if (crit->kind == ARSO_CRIT_OUTCOME || crit->kind == ARSO_CRIT_ARGMAX)
            ARSO_REQUIRE(crit->target < N, "criterion target out of range");
        if (crit->kind == ARSO_CRIT_BINNING)
            ARSO_REQUIRE(n <= NOALLOC_MAX_BINNING_QUBITS,
                         "binning without allocation supports at most 20 qubits (2^20-bit outcome bitmap)");
        cudaStream_t st = (cudaStream_t)stream;
        const NoAllocPtrs p = noalloc_setup();
        DCrit d{};
        d.kind = crit->kind;
        d.threshold = crit->threshold;
        d.target = crit->target;
        if (crit->kind == ARSO_CRIT_BINNING) {
            ARSO_REQUIRE(crit->set_len == 0 || crit->set != nullptr, "binning set is NULL");
            std::vector<uint32_t> bm((N + 31) / 32, 0);
            for (size_t i = 0; i < crit->set_len; ++i) {
                ARSO_REQUIRE(crit->set[i] < N, "binning outcome out of range");
                bm[crit->set[i] >> 5] |= 1u << (crit->set[i] & 31);
            }
            // overwrite every bitmap word this call reads (the array keeps the previous call's bits)
            ARSO_CUDA(cudaMemcpyAsync(p.bitmap, bm.data(), bm.size() * 4, cudaMemcpyHostToDevice, st));
            ARSO_CUDA(cudaStreamSynchronize(st));
            d.bitmap = p.bitmap;
        }
        const uint32_t blocks =
            launch_score_partials(amps, ref ? ref : amps, (int)n, ARSO_C64, d, p.partials, NOALLOC_MAX_BLOCKS, st);
        launch_finish_partials(p.partials, blocks, 1, nullptr, d, p.score, nullptr, st);
        ARSO_CUDA(cudaMemcpyAsync(score_out, p.score, sizeof(double), cudaMemcpyDeviceToHost, st));
        ARSO_CUDA(cudaStreamSynchronize(st));
        return ARSO_OK;
    } catch (const Error &e) {
        set_last_error(e.what());
        return e.status;
    } catch (const std::exception &e) {
        set_last_error(e.what());
        return ARSO_ECUDA;
    }
}
