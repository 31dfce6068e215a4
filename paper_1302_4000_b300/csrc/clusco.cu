// clusco.cu -- C-ABI of libclusco (see include/clusco.h). Unity build: every kernel of the
// library is included here so that the device status word lives in one translation unit.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <cstdarg>
#include <mutex>
#include <string>

#include "common.cuh"
#include "epilogue.cuh"
#include "pairs_simt.cuh"
#include "pairs_tc.cuh"
#include "prepass.cuh"
#include "vsref.cuh"
#include "backward.cuh"
#include "bwd_tc.cuh"
#include "bwd_rot.cuh"
#include "bwd_rc.cuh"
#include "drmsd.cuh"
#include "cmo.cuh"
#include "gdt.cuh"

using namespace clusco;

namespace {

thread_local std::string g_last_error;

int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

#define CUDA_TRY(call)                                                                         \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess) return fail(CLUSCO_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

inline int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }
inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Sub-buffer carving of a workspace.
struct Carver {
    char *base;
    size_t off = 0;
    explicit Carver(void *b) : base((char *)b) {}
    template <typename T>
    T *take(size_t count)
    {
        T *p = (T *)(base ? base + off : nullptr);
        off = align256(off + count * sizeof(T));
        return p;
    }
};

bool valid_form(int form)
{
    return form == CLUSCO_FORM_FP32_SIMT || form == CLUSCO_FORM_TF32 || form == CLUSCO_FORM_BF16X3 ||
           form == CLUSCO_FORM_BF16_EXACT2 || form == CLUSCO_FORM_INT_SIMT;
}

// The CUDA-core forms (no tcgen05, no rotations).
bool simt_form(int form) { return form == CLUSCO_FORM_FP32_SIMT || form == CLUSCO_FORM_INT_SIMT; }

// Layout of the all-pairs workspace; also used (with base == nullptr) to size it.
struct PairsWs {
    // SIMT (Xn: the exact-integer form's fixed-point coordinates, same layout as Xk)
    float *Xk = nullptr;
    int *Xn = nullptr;
    double *G64 = nullptr;
    // tcgen05
    void *planes = nullptr;
    float *scales = nullptr;
    float *G32 = nullptr;
    int64_t Lp = 0, Npad = 0, Rpad = 0;
    // EXACT2: the 16-bit coordinates and the mask of pairs the fast path flags
    int8_t *hplane = nullptr;
    int8_t *lplane = nullptr;
    uint32_t *flags = nullptr;
    int2 *flist = nullptr;
    int64_t flist_entries = 0;
    // rotation entry point only: the deferred-rotation list
    RotFix *fix = nullptr;
    unsigned long long *fix_count = nullptr;
    int64_t fix_cap = 0;
    size_t bytes = 0;
};

// Capacity of the deferred-rotation list: about 0.5 % of a decoy ensemble's pairs need it;
// pairs past the capacity are solved inside the forward kernel instead.
inline int64_t rotfix_cap(int64_t N)
{
    const int64_t P = N * (N - 1) / 2, cap = (int64_t)1 << 22;
    return P < cap ? P : cap;
}

PairsWs carve_pairs(void *base, int64_t N, int64_t L, int form, bool with_rot = false)
{
    PairsWs w;
    Carver c(base);
    if (form == CLUSCO_FORM_FP32_SIMT) {
        w.Lp = round_up(L, SIMT_KC);
        w.Npad = round_up(N, SIMT_TILE);
        w.Xk = c.take<float>((size_t)(w.Lp * w.Npad * 3));
        w.G64 = c.take<double>((size_t)w.Npad);
    } else if (form == CLUSCO_FORM_INT_SIMT) {
        w.Lp = round_up(L, SIMT_KC);
        w.Npad = round_up(N, SIMT_TILE);
        w.Xn = c.take<int>((size_t)(w.Lp * w.Npad * 3));
        w.scales = c.take<float>((size_t)w.Npad * 3);
        w.G64 = c.take<double>((size_t)w.Npad);
    } else {
        const int64_t kalign = (form == CLUSCO_FORM_TF32) ? 32 : 64;  // 128-byte rows
        const size_t esize = (form == CLUSCO_FORM_TF32) ? 4 : 2;
        const int nplanes = (form == CLUSCO_FORM_TF32) ? 1 : 2;
        w.Lp = round_up(L, kalign);
        w.Npad = round_up(N, TC_MA);
        w.Rpad = (w.Npad / 10) * 32;
        w.planes = c.take<char>((size_t)(nplanes * w.Rpad * w.Lp) * esize);
        w.scales = c.take<float>((size_t)w.Npad * 3);
        w.G64 = c.take<double>((size_t)w.Npad);
        w.G32 = c.take<float>((size_t)w.Npad);
        if (form == CLUSCO_FORM_BF16_EXACT2) {
            const int64_t P = N * (N - 1) / 2;
            w.hplane = c.take<int8_t>((size_t)(w.Rpad * w.Lp));
            w.lplane = c.take<int8_t>((size_t)(w.Rpad * w.Lp));
            w.flags = c.take<uint32_t>((size_t)(flag_list_offset(P) + FL_MAXSLOTS));  // mask, list counts
            w.flist_entries = flag_list_entries(P);
            w.flist = c.take<int2>((size_t)w.flist_entries);
        }
        if (with_rot) {
            w.fix_cap = rotfix_cap(N);
            w.fix = c.take<RotFix>((size_t)w.fix_cap);
            w.fix_count = c.take<unsigned long long>(1);
        }
    }
    w.bytes = c.off;
    return w;
}

int check_sizes(int64_t N, int64_t L, int64_t minN)
{
    if (N < minN) return fail(CLUSCO_EINVAL, "N=%lld must be >= %lld", (long long)N, (long long)minN);
    if (L < 1) return fail(CLUSCO_EINVAL, "L=%lld must be >= 1", (long long)L);
    if (L > (1 << 20)) return fail(CLUSCO_EINVAL, "L=%lld above the supported 2^20 atoms", (long long)L);
    if (N > (int64_t)1 << 31) return fail(CLUSCO_EOVERFLOW, "N=%lld above 2^31 models", (long long)N);
    // N*L*3 and N(N-1)/2 must fit int64 comfortably
    if ((double)N * (double)L * 3.0 > 9.0e18 || (double)N * (double)N > 9.0e18)
        return fail(CLUSCO_EOVERFLOW, "N*L*3 or N^2 overflows int64");
    return CLUSCO_OK;
}

int check_ptr(const void *p, const char *name, size_t align)
{
    if (!p) return fail(CLUSCO_EINVAL, "%s is NULL", name);
    if (((uintptr_t)p) % align) return fail(CLUSCO_EINVAL, "%s is not %zu-byte aligned", name, align);
    return CLUSCO_OK;
}

// Scratch: the caller's workspace or a stream-ordered allocation freed after use.
struct Scratch {
    void *ptr = nullptr;
    bool owned = false;
    cudaStream_t st = nullptr;
    ~Scratch()
    {
        if (owned && ptr) cudaFreeAsync(ptr, st);
    }
};

int get_scratch(Scratch &s, void *ws, size_t ws_bytes, size_t need, cudaStream_t st)
{
    s.st = st;
    if (need == 0) return CLUSCO_OK;
    if (ws) {
        if (ws_bytes < need)
            return fail(CLUSCO_ENOMEM, "workspace of %zu bytes is smaller than the %zu needed", ws_bytes, need);
        if (((uintptr_t)ws) % 256) return fail(CLUSCO_EINVAL, "workspace is not 256-byte aligned");
        s.ptr = ws;
        return CLUSCO_OK;
    }
    cudaError_t e = cudaMallocAsync(&s.ptr, need, st);
    if (e != cudaSuccess) {
        s.ptr = nullptr;
        return fail(CLUSCO_ENOMEM, "cudaMallocAsync(%zu): %s", need, cudaGetErrorString(e));
    }
    s.owned = true;
    return CLUSCO_OK;
}

int run_prepass(const float *coords, int64_t N, int64_t L, int form, const PairsWs &w, cudaStream_t st)
{
    const unsigned blocks = (unsigned)((w.Npad + 7) / 8);
    if (form == CLUSCO_FORM_FP32_SIMT) {
        prepass_simt_kernel<<<blocks, 256, 0, st>>>(coords, N, (int)L, (int)w.Lp, w.Npad, w.Xk, w.G64);
    } else if (form == CLUSCO_FORM_INT_SIMT) {
        prepass_int_kernel<<<blocks, 256, 0, st>>>(coords, N, (int)L, (int)w.Lp, w.Npad, w.Xn, w.scales, w.G64);
    } else if (form == CLUSCO_FORM_BF16_EXACT2) {
        prepass_tc_kernel<TC_EXACT2><<<blocks, 256, 0, st>>>(coords, N, (int)L, (int)w.Lp, w.Npad, w.Rpad,
                                                                w.planes, w.scales, w.G64, w.G32, nullptr, w.hplane,
                                                                w.lplane);
    } else if (form == CLUSCO_FORM_BF16X3) {
        prepass_tc_kernel<TC_BF16X3><<<blocks, 256, 0, st>>>(coords, N, (int)L, (int)w.Lp, w.Npad, w.Rpad,
                                                                w.planes, w.scales, w.G64, w.G32, nullptr);
    } else {
        prepass_tc_kernel<TC_TF32><<<blocks, 256, 0, st>>>(coords, N, (int)L, (int)w.Lp, w.Npad, w.Rpad,
                                                              w.planes, w.scales, w.G64, w.G32, nullptr);
    }
    CUDA_TRY(cudaGetLastError());
    return CLUSCO_OK;
}

// Threshold mode of the all-pairs call: the pairs with c < tau as a list (see PairSink).
struct Threshold {
    long long *list;
    float *vals;
    unsigned long long *count;
    int64_t cap;
    float tau;
};

int allpairs_impl(const float *coords, int64_t N, int64_t L, int64_t row_begin, int64_t row_end, float *out,
                  int form, void *ws, size_t ws_bytes, cudaStream_t st, float *rot = nullptr,
                  const Threshold *thr = nullptr)
{
    int rc;
    if ((rc = check_sizes(N, L, 2))) return rc;
    if ((rc = check_ptr(coords, "coords", 4))) return rc;
    if (!thr && (rc = check_ptr(out, "out", 4))) return rc;
    if (!valid_form(form)) return fail(CLUSCO_EINVAL, "unknown form %d", form);
    if (rot && simt_form(form))
        return fail(CLUSCO_EUNSUPPORTED, "rotations are produced by the tensor-core forms only");
    if (form == CLUSCO_FORM_INT_SIMT && L > INT_MAX_L)
        return fail(CLUSCO_EUNSUPPORTED, "L=%lld above the 2^17 atoms of the exact-integer form", (long long)L);
    if (row_begin < 0 || row_end > N - 1 || row_begin >= row_end)
        return fail(CLUSCO_EINVAL, "row range [%lld, %lld) outside [0, N-1=%lld)", (long long)row_begin,
                    (long long)row_end, (long long)(N - 1));
    if (!simt_form(form)) {
        if ((rc = tc_supported(form, L))) return rc;
    }
    const PairsWs sized = carve_pairs(nullptr, N, L, form, rot != nullptr);
    Scratch s;
    if ((rc = get_scratch(s, ws, ws_bytes, sized.bytes, st))) return rc;
    const PairsWs w = carve_pairs(s.ptr, N, L, form, rot != nullptr);
    if ((rc = run_prepass(coords, N, L, form, w, st))) return rc;
    const int64_t out_base = condensed_idx(row_begin, row_begin + 1, N);
    if (simt_form(form)) {
        const int64_t T = w.Npad / SIMT_TILE;
        const int64_t I0 = row_begin / SIMT_TILE, I1 = (row_end - 1) / SIMT_TILE + 1;
        const int64_t t0 = tri_row_start(I0, T), nt = tri_row_start(I1, T) - t0;
        PairSink sink;
        sink.out = out;
        sink.out_base = out_base;
        if (thr) {
            sink.list = thr->list;
            sink.vals = thr->vals;
            sink.count = thr->count;
            sink.cap = thr->cap;
            sink.tau = thr->tau;
            CUDA_TRY(cudaMemsetAsync(thr->count, 0, sizeof(unsigned long long), st));
        }
        if (form == CLUSCO_FORM_INT_SIMT)
            pairs_int_kernel<<<(unsigned)(2 * nt), 256, 0, st>>>(w.Xn, w.scales, w.G64, N, w.Npad, (int)w.Lp,
                                                                 (int)L, T, t0, row_begin, row_end, sink);
        else
            pairs_simt_kernel<<<(unsigned)nt, 256, 0, st>>>(w.Xk, w.G64, N, w.Npad, (int)w.Lp, (int)L, T, t0,
                                                            row_begin, row_end, sink);
        CUDA_TRY(cudaGetLastError());
    } else {
        TcArgs a;
        a.form = form;
        a.planes = w.planes;
        a.scales = w.scales;
        a.G64 = w.G64;
        a.G32 = w.G32;
        a.N = N;
        a.L = L;
        a.Lp = w.Lp;
        a.Rpad = w.Rpad;
        a.row_begin = row_begin;
        a.row_end = row_end;
        a.out = out;
        a.out_base = out_base;
        a.rot = rot;
        a.fix = w.fix;
        a.fix_count = w.fix_count;
        a.fix_cap = w.fix_cap;
        a.flags = w.flags;
        a.flist = w.flist;
        a.flist_entries = w.flist_entries;
        a.hplane = w.hplane;
        a.lplane = w.lplane;
        if (thr) {
            a.list = thr->list;
            a.vals = thr->vals;
            a.count = thr->count;
            a.cap = thr->cap;
            a.tau = thr->tau;
        }
        std::string err;
        rc = tc_launch_allpairs(a, st, err);
        if (rc) return fail(rc, "%s", err.c_str());
    }
    return CLUSCO_OK;
}

// dRMSD workspace (see drmsd.cuh); also used (base == nullptr) to size it.
DrWs carve_drmsd(void *base, int64_t N, int64_t L, int form)
{
    DrWs w;
    Carver c(base);
    const int64_t K = L * (L - 1) / 2;
    w.Kp = round_up(K, 64);
    w.Npad = round_up(N, DR_MA);
    if (form == CLUSCO_FORM_BF16_EXACT2)
        w.planes = c.take<char>((size_t)(2 * w.Npad * w.Kp) * 2);
    else
        w.planes = c.take<float>((size_t)(w.Npad * w.Kp));
    w.S = c.take<long long>((size_t)w.Npad);
    w.fin = c.take<int>((size_t)N);
    w.dmax = c.take<unsigned>(1);
    w.ntiles = dr_ntiles(w.Npad / DR_MA, w.Npad / DR_MB);
    if (form == CLUSCO_FORM_BF16_EXACT2) w.tiles = c.take<int2>((size_t)w.ntiles);
    w.bytes = c.off;
    return w;
}

bool drmsd_form(int form) { return form == CLUSCO_FORM_FP32_SIMT || form == CLUSCO_FORM_BF16_EXACT2; }

// Contact-map workspace (see cmo.cuh); also used (base == nullptr) to size it. K is padded to
// 1024 so that the bit-packed rows hold whole 32-word slabs.
CmWs carve_cmo(void *base, int64_t N, int64_t L, int form)
{
    CmWs w;
    Carver c(base);
    const int64_t K = L * (L - 1) / 2;
    w.Kp = round_up(K, 1024);
    w.Npad = round_up(N, CM_MB);
    w.map = c.take<uint8_t>((size_t)(w.Npad * w.Kp));
    w.cnt = c.take<int>((size_t)w.Npad);
    if (form == CLUSCO_FORM_FP8_EXACT) {
        w.ntiles = cm_ntiles(w.Npad / CM_MA, w.Npad / CM_MB);
        w.tiles = c.take<int2>((size_t)w.ntiles);
    } else {
        w.bits = c.take<uint32_t>((size_t)(w.Npad * (w.Kp / 32)));
    }
    w.bytes = c.off;
    return w;
}

bool cmo_form(int form) { return form == CLUSCO_FORM_FP32_SIMT || form == CLUSCO_FORM_FP8_EXACT; }

}  // namespace

extern "C" {

int clusco_version(void) { return 10000; }

const char *clusco_last_error(void) { return g_last_error.c_str(); }

size_t clusco_workspace_bytes(int op, int64_t N, int64_t L, int form)
{
    if (N < 1 || L < 1 || L > (1 << 20)) return 0;
    if (op == CLUSCO_OP_ALLPAIRS) {
        if (!valid_form(form) || N < 2) return 0;
        return carve_pairs(nullptr, N, L, form).bytes;
    }
    if (op == CLUSCO_OP_VS_REF) {
        Carver c(nullptr);
        c.take<int>((size_t)L * 3);
        c.take<RefInfo>(1);
        return c.off;
    }
    if (op == CLUSCO_OP_BACKWARD) {
        if (!valid_form(form) || N < 2) return 0;
        return backward_ws_bytes(N, L, form);
    }
    if (op == CLUSCO_OP_ALLPAIRS_ROT) {
        if (!valid_form(form) || simt_form(form) || N < 2) return 0;
        return carve_pairs(nullptr, N, L, form, true).bytes;
    }
    if (op == CLUSCO_OP_BACKWARD_ROT) {
        if (N < 2 || !bwr_supported(L)) return 0;
        return carve_bt(nullptr, N, L).bytes;
    }
    if (op == CLUSCO_OP_DRMSD) {
        if (!drmsd_form(form) || N < 2 || L < 2 || L > DR_MAX_L) return 0;
        return carve_drmsd(nullptr, N, L, form).bytes;
    }
    if (op == CLUSCO_OP_CMO) {
        if (!cmo_form(form) || N < 2 || L < 2 || L > DR_MAX_L) return 0;
        return carve_cmo(nullptr, N, L, form).bytes;
    }
    if (op == CLUSCO_OP_STEP) {
        if (!valid_form(form) || simt_form(form) || N < 2 || !rc_supported(L)) return 0;
        return align256(carve_pairs(nullptr, N, L, form).bytes) + carve_rc(nullptr, N, L).bytes;
    }
    if (op == CLUSCO_OP_STEP_ROT) {
        if (!valid_form(form) || simt_form(form) || N < 2 || !bwr_supported(L)) return 0;
        return align256(carve_pairs(nullptr, N, L, form, true).bytes) + carve_bt(nullptr, N, L).bytes;
    }
    return 0;
}

int clusco_crmsd_allpairs(const float *coords, int64_t N, int64_t L, float *out, int form, void *workspace,
                          size_t workspace_bytes, void *stream)
{
    g_last_error.clear();
    if (N < 2) return fail(CLUSCO_EINVAL, "N=%lld must be >= 2", (long long)N);
    return allpairs_impl(coords, N, L, 0, N - 1, out, form, workspace, workspace_bytes, (cudaStream_t)stream);
}

int clusco_crmsd_allpairs_panel(const float *coords, int64_t N, int64_t L, int64_t row_begin, int64_t row_end,
                                float *out_panel, int form, void *workspace, size_t workspace_bytes, void *stream)
{
    g_last_error.clear();
    return allpairs_impl(coords, N, L, row_begin, row_end, out_panel, form, workspace, workspace_bytes,
                         (cudaStream_t)stream);
}

int clusco_crmsd_allpairs_below(const float *coords, int64_t N, int64_t L, float tau, int64_t *list, float *vals,
                                int64_t cap, uint64_t *count, int form, void *workspace, size_t workspace_bytes,
                                void *stream)
{
    g_last_error.clear();
    int rc;
    if (tau != tau) return fail(CLUSCO_EINVAL, "tau is NaN");
    if (cap < 0) return fail(CLUSCO_EINVAL, "cap=%lld must be >= 0", (long long)cap);
    if (cap > 0) {
        if ((rc = check_ptr(list, "list", 8))) return rc;
        if ((rc = check_ptr(vals, "vals", 4))) return rc;
    }
    if ((rc = check_ptr(count, "count", 8))) return rc;
    static_assert(sizeof(int64_t) == sizeof(long long) && sizeof(uint64_t) == sizeof(unsigned long long), "");
    const Threshold t{reinterpret_cast<long long *>(list), vals, reinterpret_cast<unsigned long long *>(count), cap,
                      tau};
    return allpairs_impl(coords, N, L, 0, N - 1, nullptr, form, workspace, workspace_bytes, (cudaStream_t)stream,
                         nullptr, &t);
}

int clusco_drmsd_allpairs(const float *coords, int64_t N, int64_t L, float *out, int form, void *workspace,
                          size_t workspace_bytes, void *stream)
{
    g_last_error.clear();
    int rc;
    if ((rc = check_sizes(N, L, 2))) return rc;
    if (L < 2) return fail(CLUSCO_EINVAL, "L=%lld: dRMSD needs at least one atom pair", (long long)L);
    if (L > DR_MAX_L) return fail(CLUSCO_EINVAL, "dRMSD supports L <= %d", DR_MAX_L);
    if (N > (int64_t)1 << 24) return fail(CLUSCO_EINVAL, "dRMSD supports N <= 2^24 models");
    if ((rc = check_ptr(coords, "coords", 4))) return rc;
    if ((rc = check_ptr(out, "out", 4))) return rc;
    if (!drmsd_form(form)) return fail(CLUSCO_EUNSUPPORTED, "dRMSD forms: FP32_SIMT and BF16_EXACT2 (got %d)", form);
    if (form == CLUSCO_FORM_BF16_EXACT2 && (rc = tc_supported(CLUSCO_FORM_BF16X3, L)))
        return fail(rc, "the tensor-core dRMSD form needs an sm_103 device");
    cudaStream_t st = (cudaStream_t)stream;
    const DrWs sized = carve_drmsd(nullptr, N, L, form);
    Scratch s;
    if ((rc = get_scratch(s, workspace, workspace_bytes, sized.bytes, st))) return rc;
    const DrWs w = carve_drmsd(s.ptr, N, L, form);
    std::string err;
    rc = drmsd_launch(coords, N, L, out, form == CLUSCO_FORM_BF16_EXACT2, w, st, err);
    if (rc) return fail(rc, "%s", err.c_str());
    return CLUSCO_OK;
}

int clusco_cmo_allpairs(const float *coords, int64_t N, int64_t L, float cutoff, float *out, int form,
                        void *workspace, size_t workspace_bytes, void *stream)
{
    g_last_error.clear();
    int rc;
    if ((rc = check_sizes(N, L, 2))) return rc;
    if (L < 2) return fail(CLUSCO_EINVAL, "L=%lld: a contact map needs at least one atom pair", (long long)L);
    if (L > DR_MAX_L) return fail(CLUSCO_EINVAL, "the contact map overlap supports L <= %d", DR_MAX_L);
    if (N > (int64_t)1 << 24) return fail(CLUSCO_EINVAL, "the contact map overlap supports N <= 2^24 models");
    if (!(cutoff > 0.f) || !std::isfinite(cutoff)) return fail(CLUSCO_EINVAL, "cutoff must be positive and finite");
    if ((rc = check_ptr(coords, "coords", 4))) return rc;
    if ((rc = check_ptr(out, "out", 4))) return rc;
    if (!cmo_form(form))
        return fail(CLUSCO_EUNSUPPORTED, "contact map overlap forms: FP32_SIMT and FP8_EXACT (got %d)", form);
    if (form == CLUSCO_FORM_FP8_EXACT && (rc = tc_supported(CLUSCO_FORM_BF16X3, L)))
        return fail(rc, "the tensor-core contact map form needs an sm_103 device");
    cudaStream_t st = (cudaStream_t)stream;
    const CmWs sized = carve_cmo(nullptr, N, L, form);
    Scratch s;
    if ((rc = get_scratch(s, workspace, workspace_bytes, sized.bytes, st))) return rc;
    const CmWs w = carve_cmo(s.ptr, N, L, form);
    std::string err;
    rc = cmo_launch(coords, N, L, cutoff, out, form == CLUSCO_FORM_FP8_EXACT, w, st, err);
    if (rc) return fail(rc, "%s", err.c_str());
    return CLUSCO_OK;
}

int clusco_gdt_tm_vs_ref(const float *coords, int64_t N, int64_t L, const float *ref, float *out, void *stream)
{
    g_last_error.clear();
    int rc;
    if ((rc = check_sizes(N, L, 1))) return rc;
    if (L < 3 || L > GT_MAX_L) return fail(CLUSCO_EINVAL, "GDT_TS / TM-score need 3 <= L <= %d", GT_MAX_L);
    if (N > ((int64_t)1 << 31) - 1) return fail(CLUSCO_EINVAL, "N=%lld above one block per model", (long long)N);
    if ((rc = check_ptr(coords, "coords", 4))) return rc;
    if ((rc = check_ptr(ref, "ref", 4))) return rc;
    if ((rc = check_ptr(out, "out", 4))) return rc;
    std::string err;
    rc = gdt_tm_launch(coords, N, L, ref, out, (cudaStream_t)stream, err);
    if (rc) return fail(rc, "%s", err.c_str());
    return CLUSCO_OK;
}

int clusco_crmsd_vs_ref(const float *coords, int64_t N, int64_t L, const float *ref, float *out, void *workspace,
                        size_t workspace_bytes, void *stream)
{
    g_last_error.clear();
    int rc;
    if ((rc = check_sizes(N, L, 1))) return rc;
    if ((rc = check_ptr(coords, "coords", 4))) return rc;
    if ((rc = check_ptr(ref, "ref", 4))) return rc;
    if ((rc = check_ptr(out, "out", 4))) return rc;
    if (L > 18000) return fail(CLUSCO_EINVAL, "vs_ref supports L <= 18000 (reference staged in shared memory)");
    cudaStream_t st = (cudaStream_t)stream;
    Scratch s;
    const size_t need = clusco_workspace_bytes(CLUSCO_OP_VS_REF, N, L, 0);
    if ((rc = get_scratch(s, workspace, workspace_bytes, need, st))) return rc;
    Carver c(s.ptr);
    int *nref = c.take<int>((size_t)L * 3);
    RefInfo *info = c.take<RefInfo>(1);
    ref_prepass_kernel<<<1, RP_THREADS, 0, st>>>(ref, (int)L, nref, info);
    CUDA_TRY(cudaGetLastError());
    const size_t smem = (size_t)L * 3 * sizeof(int);
    if (smem > 48 * 1024) CUDA_TRY(cudaFuncSetAttribute(vsref_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    vsref_kernel<<<(unsigned)((N + VSREF_MODELS - 1) / VSREF_MODELS), 256, smem, st>>>(coords, N, (int)L, nref, info, out);
    CUDA_TRY(cudaGetLastError());
    return CLUSCO_OK;
}

int clusco_crmsd_allpairs_backward(const float *coords, int64_t N, int64_t L, const float *grad_out,
                                   const float *crmsd, float *grad_coords, float eps, int form, void *workspace,
                                   size_t workspace_bytes, void *stream)
{
    g_last_error.clear();
    int rc;
    if ((rc = check_sizes(N, L, 2))) return rc;
    if ((rc = check_ptr(coords, "coords", 4))) return rc;
    if ((rc = check_ptr(grad_out, "grad_out", 4))) return rc;
    if ((rc = check_ptr(crmsd, "crmsd", 4))) return rc;
    if ((rc = check_ptr(grad_coords, "grad_coords", 4))) return rc;
    if (!(eps > 0.f) || !std::isfinite(eps)) return fail(CLUSCO_EINVAL, "eps=%g must be finite and > 0", (double)eps);
    if (!valid_form(form)) return fail(CLUSCO_EINVAL, "unknown form %d", form);
    cudaStream_t st = (cudaStream_t)stream;
    Scratch s;
    const size_t need = backward_ws_bytes(N, L, form);
    if ((rc = get_scratch(s, workspace, workspace_bytes, need, st))) return rc;
    std::string err;
    rc = backward_launch(coords, N, L, grad_out, crmsd, grad_coords, eps, form, s.ptr, st, err);
    if (rc) return fail(rc, "%s", err.c_str());
    return CLUSCO_OK;
}

int clusco_crmsd_allpairs_rot(const float *coords, int64_t N, int64_t L, float *out, float *rot, int form,
                              void *workspace, size_t workspace_bytes, void *stream)
{
    g_last_error.clear();
    if (N < 2) return fail(CLUSCO_EINVAL, "N=%lld must be >= 2", (long long)N);
    int rc;
    if ((rc = check_ptr(rot, "rot", 16))) return rc;
    return allpairs_impl(coords, N, L, 0, N - 1, out, form, workspace, workspace_bytes, (cudaStream_t)stream, rot);
}

int clusco_crmsd_allpairs_backward_rot(const float *coords, int64_t N, int64_t L, const float *grad_out,
                                       const float *crmsd, const float *rot, float *grad_coords, float eps,
                                       void *workspace, size_t workspace_bytes, void *stream)
{
    g_last_error.clear();
    int rc;
    if ((rc = check_sizes(N, L, 2))) return rc;
    if ((rc = check_ptr(coords, "coords", 4))) return rc;
    if ((rc = check_ptr(grad_out, "grad_out", 4))) return rc;
    if ((rc = check_ptr(crmsd, "crmsd", 4))) return rc;
    if ((rc = check_ptr(rot, "rot", 16))) return rc;
    if ((rc = check_ptr(grad_coords, "grad_coords", 4))) return rc;
    if (!(eps > 0.f) || !std::isfinite(eps)) return fail(CLUSCO_EINVAL, "eps=%g must be finite and > 0", (double)eps);
    if (!bwr_supported(L)) return fail(CLUSCO_EUNSUPPORTED, "L=%lld above the 512 atoms of this path", (long long)L);
    if ((rc = tc_supported(CLUSCO_FORM_BF16_EXACT2, L))) return fail(rc, "tensor-core path unavailable on this device");
    cudaStream_t st = (cudaStream_t)stream;
    Scratch s;
    const size_t need = carve_bt(nullptr, N, L).bytes;
    if ((rc = get_scratch(s, workspace, workspace_bytes, need, st))) return rc;
    std::string err;
    rc = bwr_launch(coords, N, L, grad_out, crmsd, rot, grad_coords, eps, s.ptr, st, err);
    if (rc) return fail(rc, "%s", err.c_str());
    return CLUSCO_OK;
}

}  // extern "C"

// ---- one-versus-reference without device allocation --------------------------
// The scratch of clusco_crmsd_vs_ref_noalloc: the quantised reference (3 int32 per atom)
// followed by its RefInfo. In host code g_vsref_scratch only names the symbol; its device
// address is looked up on every call with cudaGetSymbolAddress (a host-side lookup once the
// module is loaded), so that it is never stale: after a cudaDeviceReset the module is loaded
// again and the symbol may move.
namespace {
constexpr size_t NOALLOC_REF_BYTES = ((size_t)CLUSCO_NOALLOC_MAX_L * 3 * sizeof(int) + 255) & ~(size_t)255;
}  // namespace

static __device__ __align__(256) unsigned char g_vsref_scratch[NOALLOC_REF_BYTES + 256];

namespace {
// Device address of g_vsref_scratch in the current context.
int noalloc_scratch(void **out)
{
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_vsref_scratch);
    if (e != cudaSuccess || !p)
        return fail(CLUSCO_ECUDA, "cudaGetSymbolAddress(g_vsref_scratch): %s", cudaGetErrorString(e));
    *out = p;
    return CLUSCO_OK;
}
}  // namespace

extern "C" {

int clusco_crmsd_vs_ref_noalloc(const float *coords, int64_t N, int64_t L, const float *ref, float *out, void *stream)
{
    g_last_error.clear();
    int rc;
    if ((rc = check_sizes(N, L, 1))) return rc;
    if ((rc = check_ptr(coords, "coords", 4))) return rc;
    if ((rc = check_ptr(ref, "ref", 4))) return rc;
    if ((rc = check_ptr(out, "out", 4))) return rc;
    if (L > CLUSCO_NOALLOC_MAX_L)
        return fail(CLUSCO_EINVAL, "L=%lld exceeds the %d-atom maximum of the no-allocation entry point",
                    (long long)L, CLUSCO_NOALLOC_MAX_L);
    void *scratch = nullptr;
    if ((rc = noalloc_scratch(&scratch))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    int *nref = (int *)scratch;
    RefInfo *info = (RefInfo *)((char *)scratch + NOALLOC_REF_BYTES);
    ref_prepass_kernel<<<1, RP_THREADS, 0, st>>>(ref, (int)L, nref, info);
    CUDA_TRY(cudaGetLastError());
    const size_t smem = (size_t)L * 3 * sizeof(int);
    if (smem > 48 * 1024) CUDA_TRY(cudaFuncSetAttribute(vsref_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    vsref_kernel<<<(unsigned)((N + VSREF_MODELS - 1) / VSREF_MODELS), 256, smem, st>>>(coords, N, (int)L, nref, info, out);
    CUDA_TRY(cudaGetLastError());
    return CLUSCO_OK;
}

int clusco_profile_enable(int on)
{
    g_last_error.clear();
    clusco::ProfState &p = clusco::prof_state();
    std::lock_guard<std::mutex> g(p.m);
    if (on) {  // a fresh window: drop whatever an earlier window left unread
        for (auto &v : p.ev) {
            for (cudaEvent_t e : v) cudaEventDestroy(e);
            v.clear();
        }
    }
    p.on.store(on != 0);
    return CLUSCO_OK;
}

int clusco_profile_read(int kernel, double *total_ms, long long *launches)
{
    g_last_error.clear();
    if (kernel < 0 || kernel >= clusco::PROF_KINDS || !total_ms || !launches)
        return fail(CLUSCO_EINVAL, "clusco_profile_read: bad kernel id or null output");
    clusco::ProfState &p = clusco::prof_state();
    std::lock_guard<std::mutex> g(p.m);
    std::vector<cudaEvent_t> &v = p.ev[kernel];
    double tot = 0.0;
    long long n = 0;
    int rc = CLUSCO_OK;
    for (size_t i = 0; i + 1 < v.size(); i += 2) {
        float ms = 0.f;
        cudaError_t e = cudaEventSynchronize(v[i + 1]);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, v[i], v[i + 1]);
        if (e != cudaSuccess) {
            rc = fail(CLUSCO_ECUDA, "clusco_profile_read: %s", cudaGetErrorString(e));
            break;
        }
        tot += ms;
        ++n;
    }
    for (cudaEvent_t e : v) cudaEventDestroy(e);
    v.clear();
    *total_ms = tot;
    *launches = n;
    return rc;
}

#ifdef CLUSCO_DEBUG_HOOKS
int clusco_debug_hooks(int skip_arrive, int64_t nd_cap)
{
    g_last_error.clear();
    if (nd_cap < 0) return fail(CLUSCO_EINVAL, "nd_cap=%lld must be >= 0", (long long)nd_cap);
    const int v = skip_arrive ? 1 : 0;
    CUDA_TRY(cudaMemcpyToSymbol(g_debug_skip_arrive, &v, sizeof v));
    debug_nd_cap() = nd_cap;
    return CLUSCO_OK;
}

int clusco_debug_flag_list_cap(int cap)
{
    g_last_error.clear();
    if (cap < 0) return fail(CLUSCO_EINVAL, "cap=%d must be >= 0", cap);
    debug_fl_cap() = cap;
    return CLUSCO_OK;
}
#endif

int clusco_sync_status(void *stream)
{
    g_last_error.clear();
    CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    unsigned int st = 0, zero = 0;
    CUDA_TRY(cudaMemcpyFromSymbol(&st, g_clusco_status, sizeof st));
    CUDA_TRY(cudaMemcpyToSymbol(g_clusco_status, &zero, sizeof zero));
    if (st & CLUSCO_ST_TIMEOUT) return fail(CLUSCO_ETIMEOUT, "a bounded device wait gave up (status 0x%x)", st);
    if (st & CLUSCO_ST_NONFINITE) return fail(CLUSCO_ENONFINITE, "non-finite input coordinate (status 0x%x)", st);
    if (st & CLUSCO_ST_BOUNDS) return fail(CLUSCO_ECUDA, "device bounds check fired (status 0x%x)", st);
    return CLUSCO_OK;
}

}  // extern "C"

// ---- one training step in one call ------------------------------------------------------
// The adjoint's pre-pass reads only the coordinates and the weights, so the fused steps run it on
// a stream of the library's own, forked from and joined back into the caller's stream by events
// of the call, while the forward runs on the caller's stream. Every host thread has its own side
// stream per device (created on the thread's first fused call on that device, kept until the
// process exits), so that calls from different threads, captured into a graph or not, never
// share one.
namespace {
constexpr int SIDE_MAX_DEVICES = 64;
thread_local cudaStream_t t_side[SIDE_MAX_DEVICES] = {};

int side_stream(cudaStream_t *out)
{
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= SIDE_MAX_DEVICES) return fail(CLUSCO_EUNSUPPORTED, "device %d beyond the side-stream table", dev);
    if (!t_side[dev]) CUDA_TRY(cudaStreamCreateWithFlags(&t_side[dev], cudaStreamNonBlocking));
    *out = t_side[dev];
    return CLUSCO_OK;
}

// The call's two events, destroyed when it returns (the runtime keeps an event alive until the
// work that records or waits on it has been enqueued).
struct EventPair {
    cudaEvent_t fork = nullptr, join = nullptr;
    ~EventPair()
    {
        if (fork) cudaEventDestroy(fork);
        if (join) cudaEventDestroy(join);
    }
};

// The fused step: prepare(side) beside forward(stream), then the join, then sweep(stream). The join
// is recorded whatever happened, so that stream never waits on an unrecorded event, and stream
// waits on it before anything that follows (the sweep, and on every return the stream-ordered free
// of a workspace the call allocated). Should recording the join itself fail, stream cannot be
// ordered after the side stream: outside a capture the call then synchronises the side stream;
// inside one it returns the error (the capture is invalid anyway).
template <typename Prep, typename Fwd, typename Sweep>
int fused_step(cudaStream_t st, Prep prepare, Fwd forward, Sweep sweep)
{
    cudaStream_t side = nullptr;
    int rc;
    if ((rc = side_stream(&side))) return rc;
    EventPair ev;
    CUDA_TRY(cudaEventCreateWithFlags(&ev.fork, cudaEventDisableTiming));
    CUDA_TRY(cudaEventCreateWithFlags(&ev.join, cudaEventDisableTiming));
    // fork: the pre-pass after everything already on stream (its inputs, the workspace)
    CUDA_TRY(cudaEventRecord(ev.fork, st));
    CUDA_TRY(cudaStreamWaitEvent(side, ev.fork, 0));
    std::string err;
    rc = prepare(side, err);
    const cudaError_t ej = cudaEventRecord(ev.join, side);
    if (rc == CLUSCO_OK && ej == cudaSuccess)
        rc = forward();
    else if (rc)
        rc = fail(rc, "%s", err.c_str());
    else
        rc = fail(CLUSCO_ECUDA, "cudaEventRecord (join): %s", cudaGetErrorString(ej));
    cudaError_t ew;
    if (ej == cudaSuccess) {
        ew = cudaStreamWaitEvent(st, ev.join, 0);
    } else {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        ew = cudaStreamIsCapturing(side, &cs);
        if (ew == cudaSuccess && cs == cudaStreamCaptureStatusNone) ew = cudaStreamSynchronize(side);
    }
    if (rc) return rc;
    if (ew != cudaSuccess) return fail(CLUSCO_ECUDA, "join of the side stream: %s", cudaGetErrorString(ew));
    rc = sweep(err);
    if (rc) return fail(rc, "%s", err.c_str());
    return CLUSCO_OK;
}
}  // namespace

extern "C" {

int clusco_crmsd_allpairs_step_rot(const float *coords, int64_t N, int64_t L, const float *grad_out, float *out,
                                   float *rot, float *grad_coords, int form, float eps, void *workspace,
                                   size_t workspace_bytes, void *stream)
{
    g_last_error.clear();
    int rc;
    if ((rc = check_sizes(N, L, 2))) return rc;
    if ((rc = check_ptr(coords, "coords", 4))) return rc;
    if ((rc = check_ptr(grad_out, "grad_out", 4))) return rc;
    if ((rc = check_ptr(out, "out", 4))) return rc;
    if ((rc = check_ptr(rot, "rot", 16))) return rc;
    if ((rc = check_ptr(grad_coords, "grad_coords", 4))) return rc;
    if (!valid_form(form)) return fail(CLUSCO_EINVAL, "unknown form %d", form);
    if (simt_form(form))
        return fail(CLUSCO_EUNSUPPORTED, "rotations are produced by the tensor-core forms only");
    if (!(eps > 0.f) || !std::isfinite(eps)) return fail(CLUSCO_EINVAL, "eps=%g must be finite and > 0", (double)eps);
    if (!bwr_supported(L)) return fail(CLUSCO_EUNSUPPORTED, "L=%lld above the 512 atoms of this path", (long long)L);
    if ((rc = tc_supported(CLUSCO_FORM_BF16_EXACT2, L))) return fail(rc, "tensor-core path unavailable on this device");
    if ((rc = tc_supported(form, L))) return fail(rc, "tensor-core path unavailable for form %d", form);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t fwd_bytes = align256(carve_pairs(nullptr, N, L, form, true).bytes);
    const size_t need = fwd_bytes + carve_bt(nullptr, N, L).bytes;
    Scratch s;
    if ((rc = get_scratch(s, workspace, workspace_bytes, need, st))) return rc;
    void *ws_bwd = static_cast<unsigned char *>(s.ptr) + fwd_bytes;
    return fused_step(
        st, [&](cudaStream_t side, std::string &err) { return bwr_prepare(coords, N, L, grad_out, ws_bwd, side, err); },
        [&]() { return allpairs_impl(coords, N, L, 0, N - 1, out, form, s.ptr, fwd_bytes, st, rot); },
        [&](std::string &err) {
            return bwr_sweep(coords, N, L, grad_out, out, rot, grad_coords, eps, ws_bwd, st, err);
        });
}

int clusco_crmsd_allpairs_step(const float *coords, int64_t N, int64_t L, const float *grad_out, float *out,
                               float *grad_coords, int form, float eps, void *workspace, size_t workspace_bytes,
                               void *stream)
{
    g_last_error.clear();
    int rc;
    if ((rc = check_sizes(N, L, 2))) return rc;
    if ((rc = check_ptr(coords, "coords", 4))) return rc;
    if ((rc = check_ptr(grad_out, "grad_out", 4))) return rc;
    if ((rc = check_ptr(out, "out", 4))) return rc;
    if ((rc = check_ptr(grad_coords, "grad_coords", 4))) return rc;
    if (!valid_form(form)) return fail(CLUSCO_EINVAL, "unknown form %d", form);
    if (simt_form(form)) return fail(CLUSCO_EUNSUPPORTED, "the fused step needs a tensor-core form");
    if (!(eps > 0.f) || !std::isfinite(eps)) return fail(CLUSCO_EINVAL, "eps=%g must be finite and > 0", (double)eps);
    if (!rc_supported(L)) return fail(CLUSCO_EUNSUPPORTED, "L=%lld above the 1024 atoms of this path", (long long)L);
    if ((rc = tc_supported(CLUSCO_FORM_BF16_EXACT2, L))) return fail(rc, "tensor-core path unavailable on this device");
    if ((rc = tc_supported(form, L))) return fail(rc, "tensor-core path unavailable for form %d", form);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t fwd_bytes = align256(carve_pairs(nullptr, N, L, form).bytes);
    const size_t need = fwd_bytes + carve_rc(nullptr, N, L).bytes;
    Scratch s;
    if ((rc = get_scratch(s, workspace, workspace_bytes, need, st))) return rc;
    void *ws_bwd = static_cast<unsigned char *>(s.ptr) + fwd_bytes;
    return fused_step(
        st, [&](cudaStream_t side, std::string &err) { return rc_prepare(coords, N, L, grad_out, ws_bwd, side, err); },
        [&]() { return allpairs_impl(coords, N, L, 0, N - 1, out, form, s.ptr, fwd_bytes, st); },
        [&](std::string &err) { return rc_sweep(coords, N, L, grad_out, out, grad_coords, eps, ws_bwd, st, err); });
}

}  // extern "C"
