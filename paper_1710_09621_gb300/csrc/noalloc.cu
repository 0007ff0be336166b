// odwf_apply_noalloc: the D_T / H_T apply of odwf_apply for callers that must not allocate
// device memory during the call.
//
// Who needs it: code that runs where cudaMalloc is unavailable or forbidden after start-up, such
// as a caller that has handed all device memory to its own pool or arena, a process whose memory
// budget is fixed once at initialisation, or a step that must not touch the allocator between
// two synchronisation points. odwf_apply allocates its even-odd work fields and the per-mass-pair
// coefficient block on first use; this entry point instead uses one file-scope device array.
//
// The array is kScratchBytes (32 MiB) of static device memory. Every GPU that loads the library
// holds it until the process exits. It must hold four even-odd half fields of the requested
// precision plus the fifth-dimension coefficients, which limits Vh * Ns (checkerboard sites times
// slices) to about 43,000 in FP64 and 87,000 in FP32; larger lattices are rejected with
// ODWF_EINVAL. All calls share the array: two calls whose GPU work overlaps (different streams or
// threads without ordering) race on it, and each call overwrites every byte it reads before
// reading it, so nothing left by an earlier call is used.
#include <cstdio>
#include <string>
#include <vector>

#include "odwf_internal.h"

namespace {

constexpr size_t kScratchBytes = size_t(32) << 20;
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_apply_scratch[kScratchBytes];

// Device address of g_apply_scratch per device, set on the first call made with that device
// current. (In host code the symbol is only a host-side stand-in, never a device address.)
void* g_scratch_addr[kMaxDevices] = {nullptr};

inline size_t round256(size_t b) { return (b + 255) & ~size_t(255); }

}  // namespace

extern "C" int odwf_apply_noalloc(odwf_t* h, int op, double m1, double m2, const void* in, void* out, int prec,
                                  void* stream) {
    using namespace odwf;
    if (!h || !in || !out) return set_err(h, ODWF_EINVAL, "null argument");
    if (!h->have_gauge) return set_err(h, ODWF_EINVAL, "odwf_set_gauge has not been called");
    if (op != ODWF_OP_DT && op != ODWF_OP_HT) return set_err(h, ODWF_EINVAL, "odwf_apply_noalloc: op must be DT or HT");
    if (prec != ODWF_PREC_DOUBLE && prec != ODWF_PREC_SINGLE)
        return set_err(h, ODWF_EINVAL, "odwf_apply_noalloc: prec must be DOUBLE or SINGLE");
    if (!(m1 > 0.0 && m1 <= 1.0) || !(m2 > 0.0 && m2 <= 1.0)) return set_err(h, ODWF_EINVAL, "masses must lie in (0, 1]");
    cudaStream_t st = (cudaStream_t)stream;
    const int stg = prec == ODWF_PREC_DOUBLE ? ST_DOUBLE : ST_FLOAT;

    const size_t field = round256(half_elems_bytes(h, stg));
    const size_t coef_bytes = round256(sizeof(double) * kNumCoef * h->Ns * h->Ns);
    const size_t need = 4 * field + coef_bytes;
    if (need > kScratchBytes) {
        return set_err(h, ODWF_EINVAL,
                       "odwf_apply_noalloc: this lattice needs " + std::to_string(need) +
                           " bytes of scratch, more than the fixed maximum of " + std::to_string(kScratchBytes) +
                           " bytes; use odwf_apply");
    }
    int dev = 0;
    int rc = cuda_check(h, cudaGetDevice(&dev), "cudaGetDevice");
    if (rc) return rc;
    if (dev < 0 || dev >= kMaxDevices) return set_err(h, ODWF_EINVAL, "odwf_apply_noalloc: device index out of range");
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        rc = cuda_check(h, cudaGetSymbolAddress(&p, g_apply_scratch), "cudaGetSymbolAddress(g_apply_scratch)");
        if (rc) return rc;
        g_scratch_addr[dev] = p;
    }
    unsigned char* base = static_cast<unsigned char*>(g_scratch_addr[dev]);
    void* ie = base;
    void* io = base + field;
    void* oe = base + 2 * field;
    void* oo = base + 3 * field;
    SCoef c;
    c.dev = reinterpret_cast<double*>(base + 4 * field);

    std::vector<double> host;
    std::string err;
    if (!coef_host(h, m1, m2, host, err)) return set_err(h, ODWF_EINVAL, err);
    // pageable source: the copy is staged before the call returns, so `host` may go out of scope
    rc = cuda_check(h, cudaMemcpyAsync(c.dev, host.data(), sizeof(double) * host.size(), cudaMemcpyHostToDevice, st),
                    "coefficient copy");
    if (rc) return rc;

    const bool ht = (op == ODWF_OP_HT);
    if ((rc = launch_pack5(h, (const double*)in, ie, io, stg, 0, st))) return rc;
    if ((rc = apply_dt_parity(h, stg, &c, false, 0, io, ie, oe, st))) return rc;
    if ((rc = apply_dt_parity(h, stg, &c, false, 1, ie, io, oo, st))) return rc;
    return launch_unpack5(h, oe, oo, (double*)out, stg, ht ? 1 : 0, st);
}
