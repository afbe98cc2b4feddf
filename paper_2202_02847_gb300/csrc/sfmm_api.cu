// C ABI of the translation library: handle, argument validation, launches.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <new>
#include <vector>

#include "sfmm.h"
#include "sfmm_ctx.h"
#include "sfmm_generic.h"
#include "sfmm_kernels.cuh"
#include "sfmm_tables.h"
#include "sfmm_unrolled.cuh"
#include "sfmm_unrolled_dispatch.h"

using namespace sfmm;

static_assert(SFMM_MAX_CLASSES == MAX_CLASSES, "class table sizes of the ABI and the kernel differ");
static_assert(SFMM_MAX_PASS_CLASSES == MAX_PASS_CLASSES && SFMM_MAX_PASS_PHASES == MAX_PASS_PHASES,
              "pass table sizes of the ABI and the kernel differ");


namespace {

constexpr int kMaxPmax64 = 64;
constexpr int kMaxPmax32 = 30;

template <typename T>
void set_kernel_attrs(size_t smem) {
    set_generic_attrs<T, OP_M2M>(smem);
    set_generic_attrs<T, OP_M2L>(smem);
    set_generic_attrs<T, OP_L2L>(smem);
    set_multi_attrs<T>(smem);
    set_pass_attrs<T>(smem);
    cudaFuncSetAttribute(p2x_kernel<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(p2x_kernel<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

// Transposed copies of the swap and z-translation tables for the
// warp-cooperative kernels (layout in DevTables).
struct WideHost {
    std::vector<double> FT, GT, TzT[3];
    std::vector<int> FTrow, GTrow;
};

WideHost transpose_tables(const HostTables &ht) {
    WideHost w;
    const int P = ht.Pmax;
    for (int n = 0; n < P; ++n) {
        const int fe = n / 2 + 1, fo = (n + 1) / 2, ge = (n + 1) / 2, go = n / 2;
        w.FTrow.push_back((int)w.FT.size());
        w.GTrow.push_back((int)w.GT.size());
        const size_t f0 = w.FT.size(), g0 = w.GT.size();
        w.FT.resize(f0 + (size_t)fe * (n + 1), 0.0);
        w.GT.resize(g0 + (size_t)ge * n, 0.0);
        int fm = 0, gm = 0;                 // packed start of row m
        for (int m = 0; m <= n; ++m) {
            const int cf = ((n + m) & 1) ? fo : fe;
            for (int i = 0; i < cf; ++i) w.FT[f0 + (size_t)i * (n + 1) + m] = ht.F[ht.Frow[n] + fm + i];
            fm += cf;
            if (m >= 1) {
                const int cg = ((n + m) & 1) ? go : ge;
                for (int i = 0; i < cg; ++i) w.GT[g0 + (size_t)i * n + (m - 1)] = ht.G[ht.Grow[n] + gm + i];
                gm += cg;
            }
        }
    }
    w.FTrow.push_back((int)w.FT.size());
    w.GTrow.push_back((int)w.GT.size());
    for (int op = 0; op < 3; ++op) {
        w.TzT[op].assign(ht.Tz[op].size(), 0.0);
        for (int m = 0; m < P; ++m) {
            const long long off = ztrans_block_offset(P, m);
            const int d = P - m;
            for (int a = 0; a < d; ++a)
                for (int b = 0; b < d; ++b) w.TzT[op][off + (long long)b * d + a] = ht.Tz[op][off + (long long)a * d + b];
        }
    }
    return w;
}

// Copy the host tables (and their transposed copies) into one device buffer
// converted to T.
// M2L's swap tables with the basis factors folded in (layout of F and G):
// F diag(c), G diag(c) (first input swap) and diag(c) F, diag(c) G (last output
// swap), c_n^l = sqrt((n-l)!(n+l)!) of the row's input index l or output index m.
struct FoldedHost {
    std::vector<double> FI, GI, FO, GO;
};

FoldedHost fold_tables(const HostTables &ht) {
    FoldedHost f{ht.F, ht.G, ht.F, ht.G};
    for (int n = 0; n < ht.Pmax; ++n) {
        const double *cn = ht.c.data() + n * (n + 1) / 2;
        int i = ht.Frow[n], j = ht.Grow[n];
        for (int m = 0; m <= n; ++m) {
            for (int l = (n + m) & 1; l <= n; l += 2, ++i) {
                f.FI[i] = ht.F[i] * cn[l];
                f.FO[i] = cn[m] * ht.F[i];
            }
            if (m == 0) continue;
            for (int l = ((n + m) & 1) ? 2 : 1; l <= n; l += 2, ++j) {
                f.GI[j] = ht.G[j] * cn[l];
                f.GO[j] = cn[m] * ht.G[j];
            }
        }
    }
    return f;
}

template <typename T>
sfmm_status upload(const HostTables &ht, sfmm_ctx *h, DevTables<T> *dt) {
    const WideHost wh = transpose_tables(ht);
    constexpr bool fold = sizeof(T) == sizeof(double);
    const FoldedHost fh = fold ? fold_tables(ht) : FoldedHost{};
    const size_t nF = ht.F.size(), nG = ht.G.size(), nc = ht.c.size(), nT = ht.Tz[0].size();
    const size_t nreal = nF + nG + 2 * nc + 3 * nT + wh.FT.size() + wh.GT.size() + 3 * nT +
                         (fold ? 2 * (nF + nG) : 0);
    const size_t nint = 4 * (size_t)(ht.Pmax + 1);
    const size_t bytes = nreal * sizeof(T) + nint * sizeof(int) + 256;
    std::vector<unsigned char> host(bytes, 0);
    T *r = reinterpret_cast<T *>(host.data());
    size_t o = 0;
    auto put = [&](const std::vector<double> &v) {
        const size_t at = o;
        for (size_t i = 0; i < v.size(); ++i) r[o + i] = (T)v[i];
        o += v.size();
        return at;
    };
    // FP32: c_n^m 2^-n and 2^n / c_n^m, which stay inside the FP32 range up to
    // order 30 (the kernels multiply the row's 2^{+-n} back in, basis_factor)
    std::vector<double> cs = ht.c, ics = ht.ic;
    if (sizeof(T) == sizeof(float))
        for (int n = 0; n < ht.Pmax; ++n)
            for (int m = 0; m <= n; ++m) {
                cs[n * (n + 1) / 2 + m] = std::ldexp(ht.c[n * (n + 1) / 2 + m], -n);
                ics[n * (n + 1) / 2 + m] = std::ldexp(ht.ic[n * (n + 1) / 2 + m], n);
            }
    const size_t oF = put(ht.F), oG = put(ht.G), oc = put(cs), oic = put(ics);
    const size_t oT0 = put(ht.Tz[0]), oT1 = put(ht.Tz[1]), oT2 = put(ht.Tz[2]);
    const size_t oFT = put(wh.FT), oGT = put(wh.GT);
    const size_t oU0 = put(wh.TzT[0]), oU1 = put(wh.TzT[1]), oU2 = put(wh.TzT[2]);
    const size_t oFI = put(fh.FI), oGI = put(fh.GI), oFO = put(fh.FO), oGO = put(fh.GO);
    size_t ibyte = (o * sizeof(T) + 15) / 16 * 16;
    int *ip = reinterpret_cast<int *>(host.data() + ibyte);
    std::memcpy(ip, ht.Frow.data(), (ht.Pmax + 1) * sizeof(int));
    std::memcpy(ip + ht.Pmax + 1, ht.Grow.data(), (ht.Pmax + 1) * sizeof(int));
    std::memcpy(ip + 2 * (ht.Pmax + 1), wh.FTrow.data(), (ht.Pmax + 1) * sizeof(int));
    std::memcpy(ip + 3 * (ht.Pmax + 1), wh.GTrow.data(), (ht.Pmax + 1) * sizeof(int));
    if (cudaMalloc(&h->d_tables, bytes) != cudaSuccess) return SFMM_ERR_NOMEM;
    if (cudaMemcpy(h->d_tables, host.data(), bytes, cudaMemcpyHostToDevice) != cudaSuccess)
        return SFMM_ERR_CUDA;
    const T *d = reinterpret_cast<const T *>(h->d_tables);
    const int *di = reinterpret_cast<const int *>(static_cast<unsigned char *>(h->d_tables) + ibyte);
    dt->F = d + oF;
    dt->G = d + oG;
    dt->c = d + oc;
    dt->ic = d + oic;
    dt->Tz[0] = d + oT0;
    dt->Tz[1] = d + oT1;
    dt->Tz[2] = d + oT2;
    dt->Frow = di;
    dt->Grow = di + ht.Pmax + 1;
    dt->FT = d + oFT;
    dt->GT = d + oGT;
    dt->TzT[0] = d + oU0;
    dt->TzT[1] = d + oU1;
    dt->TzT[2] = d + oU2;
    dt->FTrow = di + 2 * (ht.Pmax + 1);
    dt->GTrow = di + 3 * (ht.Pmax + 1);
    dt->FI = fold ? d + oFI : nullptr;
    dt->GI = fold ? d + oGI : nullptr;
    dt->FO = fold ? d + oFO : nullptr;
    dt->GO = fold ? d + oGO : nullptr;
    dt->Pmax = ht.Pmax;
    return SFMM_OK;
}

// The unrolled kernels read their tables from __constant__ memory, one copy
// per module and device; fill them once per device (at the first create).
constexpr int kMaxDevices = 64;
std::mutex g_const_mu;
bool g_const_filled[kMaxDevices] = {};

sfmm_status fill_unrolled_constants(int dev, size_t smem_optin) {
    if (dev < 0 || dev >= kMaxDevices) return SFMM_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_const_mu);
    if (g_const_filled[dev]) return SFMM_OK;
    HostTables ht;
    // layout of sfmm_unrolled.cuh: packed F and G of rows n < PC, c, 1/c, the
    // three z-translation block sets and M2L's folded swaps, all built for order PC
    if (build_tables(unrolled::PC, &ht) != 0) return SFMM_ERR_ORDER;
    std::vector<double> t;
    const int nF = unrolled::FR(unrolled::PC), nG = unrolled::GR(unrolled::PC);
    t.insert(t.end(), ht.F.begin(), ht.F.begin() + nF);
    t.insert(t.end(), ht.G.begin(), ht.G.begin() + nG);
    t.insert(t.end(), ht.c.begin(), ht.c.end());
    t.insert(t.end(), ht.ic.begin(), ht.ic.end());
    for (int op = 0; op < 3; ++op) t.insert(t.end(), ht.Tz[op].begin(), ht.Tz[op].end());
    // M2L's swaps with the basis factors folded in: F diag(c), G diag(c) (first
    // input swap), then diag(c) F, diag(c) G (last output swap)
    std::vector<double> fi(nF), gi(nG), fo(nF), go(nG);
    for (int n = 0; n < unrolled::PC; ++n) {
        if (ht.Frow[n] != unrolled::FR(n) || ht.Grow[n] != unrolled::GR(n)) return SFMM_ERR_UNSUPPORTED;
        const double *cn = ht.c.data() + n * (n + 1) / 2;
        for (int m = 0; m <= n; ++m) {
            int i = unrolled::FR(n) + unrolled::FM(n, m);
            for (int l = (n + m) & 1; l <= n; l += 2, ++i) {
                fi[i] = ht.F[i] * cn[l];
                fo[i] = cn[m] * ht.F[i];
            }
            if (m == 0) continue;
            int j = unrolled::GR(n) + unrolled::GM(n, m);
            for (int l = unrolled::l0G(n, m); l <= n; l += 2, ++j) {
                gi[j] = ht.G[j] * cn[l];
                go[j] = cn[m] * ht.G[j];
            }
        }
    }
    t.insert(t.end(), fi.begin(), fi.end());
    t.insert(t.end(), gi.begin(), gi.end());
    t.insert(t.end(), fo.begin(), fo.end());
    t.insert(t.end(), go.begin(), go.end());
    if ((int)t.size() != unrolled::table_size()) return SFMM_ERR_UNSUPPORTED;
    std::vector<float> t32(t.begin(), t.end());
    if (!unrolled::fill_constants(t.data(), t32.data())) return SFMM_ERR_CUDA;
    unrolled::set_attributes(smem_optin);
    if (cudaGetLastError() != cudaSuccess) return SFMM_ERR_CUDA;
    g_const_filled[dev] = true;
    return SFMM_OK;
}

bool use_unrolled(const sfmm_ctx *h, int op, int p_in, int p_out) {
    const int pol = h->policy[op][p_in][p_out];
    if (pol != SFMM_POLICY_AUTO && pol != SFMM_POLICY_UNROLLED) return false;
    return p_in == p_out && unrolled::compiled(p_in) && h->unrolled_ok;
}

// Batch calls: AUTO takes the unrolled kernels at every compiled order but
// FP64 order 12, where the generic kernel with the rotated solid in the global
// scratch (8 warps per SM against the unrolled kernel's 5, whose solids fill
// the shared memory) is 3-10 % faster (GB300, 155,648 translations).
bool use_unrolled_batch(const sfmm_ctx *h, int op, int p_in, int p_out) {
    if (h->policy[op][p_in][p_out] == SFMM_POLICY_AUTO && h->dtype == SFMM_F64 && p_in == 12) return false;
    return use_unrolled(h, op, p_in, p_out);
}

unrolled::Launch launch_info(const sfmm_ctx *h, cudaStream_t s) {
    return unrolled::Launch{h->sm_count, h->smem_optin, h->d_status, s};
}

sfmm_status check_common(sfmm_handle h, int p_in, int p_out, long long count) {
    if (h == nullptr || count < 0) return SFMM_ERR_ARG;
    if (p_in < 1 || p_out < 1 || p_in > h->Pmax || p_out > h->Pmax) return SFMM_ERR_ORDER;
    return SFMM_OK;
}

// Launch geometry of one translation call.

template <typename T>
bool shared_only_fits(const sfmm_ctx *h, int p_in, int p_out) {
    return (size_t)(x_elems(p_in) + row_elems(p_in, p_out)) * WARP * sizeof(T) <= h->smem_optin;
}

template <typename T>
Geometry pick_geometry(const sfmm_ctx *h, int op, int p_in, int p_out, long long units) {
    Geometry g;
    const size_t sz = sizeof(T);
    const int pol = h->policy[op][p_in][p_out];
    const int wfix = h->warps[op][p_in][p_out];
    // AUTO keeps the working set in shared memory only while enough warps fit
    // per SM, else it takes the global scratch.  FP64: two blocks of at least
    // two warps (one warp per sub-partition; the FP64 pipe of a sub-partition
    // idles without one).  FP32, bound by issue and latency rather than by a
    // pipe: eight warps (below that the global scratch, cached in L1 and L2,
    // is about twice as fast on GB300 at orders 13..16).
    bool shared = pol != SFMM_POLICY_GLOBAL && shared_only_fits<T>(h, p_in, p_out);
    if (shared && pol == SFMM_POLICY_AUTO) {
        const size_t pw = (size_t)(x_elems(p_in) + row_elems(p_in, p_out)) * WARP * sz;
        const size_t slot_g = (size_t)x_elems(p_in) * WARP * sz;
        const bool global_ok = h->d_scratch != nullptr && slot_g * 4 <= h->scratch_bytes &&
                               (size_t)row_elems(p_in, p_out) * WARP * sz <= h->smem_optin;
        const bool few = sz == sizeof(float) ? h->smem_optin / pw < 8 : h->smem_optin / 2 / pw < 2;
        if (few && global_ok) shared = false;
    }
    if (shared) {
        const size_t per_warp = (size_t)(x_elems(p_in) + row_elems(p_in, p_out)) * WARP * sz;
        // aim for two resident blocks per SM (half the opt-in budget each)
        int w = (int)(h->smem_optin / 2 / per_warp);
        if (w < 1) w = 1;
        if (w > 8) w = 8;
        if (wfix > 0 && (size_t)wfix * per_warp <= h->smem_optin) w = wfix;
        g.warps = w;
        g.smem = (size_t)w * per_warp;
        g.blocks = (units + w * WARP - 1) / (w * WARP);
        return g;
    }
    const size_t per_warp = (size_t)row_elems(p_in, p_out) * WARP * sz;
    const size_t slot = (size_t)x_elems(p_in) * WARP * sz;
    if (h->d_scratch == nullptr || per_warp > h->smem_optin) return g;   // warps = 0
    int w = (int)(h->smem_optin / 2 / per_warp);
    if (w < 1) w = 1;
    if (w > 4) w = 4;
    if (wfix > 0 && (size_t)wfix * per_warp <= h->smem_optin) w = wfix;
    const long long slots = (long long)(h->scratch_bytes / slot);
    long long blocks = slots / w;
    const long long need = (units + w * WARP - 1) / (w * WARP);
    if (blocks > need) blocks = need;
    if (blocks < 1) return g;
    g.xg = true;
    g.warps = w;
    g.smem = (size_t)w * per_warp;
    g.blocks = blocks;
    return g;
}

// Order a scratch-using launch after the previous one (any stream).
struct ScratchGuard {
    sfmm_ctx *h;
    cudaStream_t s;
    bool on;
    std::unique_lock<std::mutex> lk;
    ScratchGuard(sfmm_ctx *h_, cudaStream_t s_, bool on_) : h(h_), s(s_), on(on_) {
        // inside stream capture the ordering event is skipped (a captured graph
        // replays its launches in order on its own stream)
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (on && cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
            on = false;
        if (!on) return;
        lk = std::unique_lock<std::mutex>(h->scratch_mu);
        cudaStreamWaitEvent(s, h->scratch_free, 0);
    }
    ~ScratchGuard() {
        if (on) cudaEventRecord(h->scratch_free, s);
    }
};

// The warp-cooperative kernel serves a batch call when the policy says so, or
// under AUTO where it is faster than the per-thread generic kernel (measured on
// GB300, 155,648 translations): FP32 M2L of orders 16..31 (0.78 vs 0.86 ms at
// P = 16, 3.6 vs 6.5 ms at P = 30), FP32 M2M / L2L of orders 22..31 (even at
// P = 20, 1.3x faster at P = 30), FP64 M2L of orders 30 and 31 (24.5 vs 26.8 ms
// at P = 30).  Below those orders, and for FP64 M2M / L2L, the per-thread
// kernels keep the pipes busier.
template <typename T>
bool wants_wide(const sfmm_ctx *h, int op, int p_in, int p_out) {
    const int pol = h->policy[op][p_in][p_out];
    if (pol == SFMM_POLICY_WIDE) return true;
    const int Q = p_in > p_out ? p_in : p_out;
    if (pol != SFMM_POLICY_AUTO || Q > wide_max_order()) return false;
    if (sizeof(T) == sizeof(float)) return Q >= (op == OP_M2L ? 16 : 22);
    return op == OP_M2L && Q >= 30;
}

template <typename T>
sfmm_status launch_batch(sfmm_handle h, int op, const void *const *in, void *const *out,
                         const void *shift, int p_in, int p_out, long long count,
                         int accumulate, cudaStream_t stream, const DevTables<T> &tb) {
    if (wants_wide<T>(h, op, p_in, p_out)) {
        auto I = reinterpret_cast<const T *const *>(in);
        auto O = reinterpret_cast<T *const *>(out);
        auto S = reinterpret_cast<const T *>(shift);
        const int wf = h->warps[op][p_in][p_out];
        bool ok;
        if (op == OP_M2M) ok = wide_launch<T, OP_M2M>(h, wf, stream, tb, I, O, S, p_in, p_out, count, accumulate, h->d_status);
        else if (op == OP_M2L) ok = wide_launch<T, OP_M2L>(h, wf, stream, tb, I, O, S, p_in, p_out, count, accumulate, h->d_status);
        else ok = wide_launch<T, OP_L2L>(h, wf, stream, tb, I, O, S, p_in, p_out, count, accumulate, h->d_status);
        if (ok) return cudaGetLastError() == cudaSuccess ? SFMM_OK : SFMM_ERR_CUDA;
        if (h->policy[op][p_in][p_out] == SFMM_POLICY_WIDE) return SFMM_ERR_UNSUPPORTED;
    }
    const Geometry g = pick_geometry<T>(h, op, p_in, p_out, count);
    if (g.warps < 1) return SFMM_ERR_UNSUPPORTED;
    if (g.blocks > 0x7fffffffLL) return SFMM_ERR_UNSUPPORTED;
    auto I = reinterpret_cast<const T *const *>(in);
    auto O = reinterpret_cast<T *const *>(out);
    auto S = reinterpret_cast<const T *>(shift);
    T *scr = reinterpret_cast<T *>(h->d_scratch);
    ScratchGuard guard(h, stream, g.xg);
    if (op == OP_M2M) batch_launch<T, OP_M2M>(h, g, stream, tb, I, O, S, p_in, p_out, count, accumulate, scr, h->d_status);
    else if (op == OP_M2L) batch_launch<T, OP_M2L>(h, g, stream, tb, I, O, S, p_in, p_out, count, accumulate, scr, h->d_status);
    else batch_launch<T, OP_L2L>(h, g, stream, tb, I, O, S, p_in, p_out, count, accumulate, scr, h->d_status);
    return cudaGetLastError() == cudaSuccess ? SFMM_OK : SFMM_ERR_CUDA;
}

// Lanes per target of the generic lists kernels when the caller does not say:
// M2L lists are long (a box's interaction list), M2M and L2L lists hold the
// eight children or the parent.
int default_lanes(int op) { return op == OP_M2L ? 32 : 8; }

// Geometry of a group-lists launch (G lanes per target, rotated solid and
// output slot per lane in the global scratch); warps = 0 if it cannot run.
template <typename T>
Geometry group_geometry(const sfmm_ctx *h, int op, int p_in, int p_out, long long n_targets, int G) {
    Geometry g;
    const size_t sz = sizeof(T);
    const size_t per_warp = (size_t)row_elems(p_in, p_out) * WARP * sz;
    const size_t slot = (size_t)(x_elems(p_in) + p_out * (p_out + 1)) * WARP * sz;
    if (h->d_scratch == nullptr || per_warp > h->smem_optin || slot > h->scratch_bytes) return g;
    int w = (int)(h->smem_optin / 2 / per_warp);
    if (w < 1) w = 1;
    if (w > 4) w = 4;
    const int wfix = h->warps[op][p_in][p_out];
    if (wfix > 0 && (size_t)wfix * per_warp <= h->smem_optin) w = wfix;
    const long long slots = (long long)(h->scratch_bytes / slot);
    if (w > slots) w = (int)slots;
    long long blocks = slots / w;
    const long long chunks = (n_targets + WARP / G - 1) / (WARP / G);
    const long long need = (chunks + w - 1) / w;
    if (blocks > need) blocks = need;
    if (blocks < 1) return g;
    g.xg = true;
    g.warps = w;
    g.smem = (size_t)w * per_warp;
    g.blocks = blocks;
    return g;
}

template <typename T>
sfmm_status launch_lists(sfmm_handle h, int op, const void *const *src, const void *shift,
                         const long long *offsets, void *const *out, int p_in, int p_out,
                         long long n_targets, int accumulate, cudaStream_t stream,
                         const DevTables<T> &tb) {
    // AUTO and GLOBAL: G lanes per target with the global scratch, if it has room
    if (h->policy[op][p_in][p_out] != SFMM_POLICY_SHARED) {
        const int G = default_lanes(op);
        const Geometry gg = group_geometry<T>(h, op, p_in, p_out, n_targets, G);
        if (gg.warps >= 1 && gg.blocks <= 0x7fffffffLL) {
            auto Sp = reinterpret_cast<const T *const *>(src);
            auto O = reinterpret_cast<T *const *>(out);
            auto S = reinterpret_cast<const T *>(shift);
            T *scr = reinterpret_cast<T *>(h->d_scratch);
            ScratchGuard guard(h, stream, true);
            if (cudaMemsetAsync(h->d_work, 0, sizeof(unsigned long long), stream) != cudaSuccess) return SFMM_ERR_CUDA;
            unsigned long long *wk = h->d_work;
            if (op == OP_M2M) glists_launch<T, OP_M2M>(h, gg, stream, tb, Sp, S, offsets, O, p_in, p_out, n_targets, accumulate, G, scr, wk, h->d_status);
            else if (op == OP_M2L) glists_launch<T, OP_M2L>(h, gg, stream, tb, Sp, S, offsets, O, p_in, p_out, n_targets, accumulate, G, scr, wk, h->d_status);
            else glists_launch<T, OP_L2L>(h, gg, stream, tb, Sp, S, offsets, O, p_in, p_out, n_targets, accumulate, G, scr, wk, h->d_status);
            return cudaGetLastError() == cudaSuccess ? SFMM_OK : SFMM_ERR_CUDA;
        }
    }
    const Geometry g = pick_geometry<T>(h, op, p_in, p_out, n_targets);
    if (g.warps < 1) return SFMM_ERR_UNSUPPORTED;
    if (g.blocks > 0x7fffffffLL) return SFMM_ERR_UNSUPPORTED;
    auto Sp = reinterpret_cast<const T *const *>(src);
    auto O = reinterpret_cast<T *const *>(out);
    auto S = reinterpret_cast<const T *>(shift);
    T *scr = reinterpret_cast<T *>(h->d_scratch);
    ScratchGuard guard(h, stream, g.xg);
    if (op == OP_M2M) lists_launch<T, OP_M2M>(h, g, stream, tb, Sp, S, offsets, O, p_in, p_out, n_targets, accumulate, scr, h->d_status);
    else if (op == OP_M2L) lists_launch<T, OP_M2L>(h, g, stream, tb, Sp, S, offsets, O, p_in, p_out, n_targets, accumulate, scr, h->d_status);
    else lists_launch<T, OP_L2L>(h, g, stream, tb, Sp, S, offsets, O, p_in, p_out, n_targets, accumulate, scr, h->d_status);
    return cudaGetLastError() == cudaSuccess ? SFMM_OK : SFMM_ERR_CUDA;
}

template <typename T>
sfmm_status launch_p2x(sfmm_handle h, bool singular, int P, const void *points, const void *q,
                       const long long *offsets, const void *centres, void *out,
                       long long n_boxes, cudaStream_t stream) {
    const size_t per_warp = (size_t)6 * P * WARP * sizeof(T);
    int w = (int)(h->smem_optin / 2 / per_warp);
    if (w < 1) w = (int)(h->smem_optin / per_warp);
    if (w < 1) return SFMM_ERR_UNSUPPORTED;
    if (w > 4) w = 4;
    const int threads = w * WARP;
    const long long blocks = (n_boxes + threads - 1) / threads;
    if (blocks > 0x7fffffffLL) return SFMM_ERR_UNSUPPORTED;
    const size_t smem = (size_t)w * per_warp;
    auto Pt = reinterpret_cast<const T *>(points);
    auto Q = reinterpret_cast<const T *>(q);
    auto C = reinterpret_cast<const T *>(centres);
    auto O = reinterpret_cast<T *>(out);
    if (singular)
        p2x_kernel<T, true><<<(unsigned)blocks, threads, smem, stream>>>(P, Pt, Q, offsets, C, O, n_boxes, h->d_status);
    else
        p2x_kernel<T, false><<<(unsigned)blocks, threads, smem, stream>>>(P, Pt, Q, offsets, C, O, n_boxes, h->d_status);
    return cudaGetLastError() == cudaSuccess ? SFMM_OK : SFMM_ERR_CUDA;
}

sfmm_status batch(sfmm_handle h, int op, const void *const *in, void *const *out,
                  const void *shift, int p_in, int p_out, long long count, int accumulate,
                  sfmm_stream stream) {
    sfmm_status st = check_common(h, p_in, p_out, count);
    if (st != SFMM_OK) return st;
    if (count == 0) return SFMM_OK;
    if (in == nullptr || out == nullptr || shift == nullptr) return SFMM_ERR_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (use_unrolled_batch(h, op, p_in, p_out))
        return unrolled::launch_batch(h->dtype == SFMM_F64, p_in, op, in, out, shift, count,
                                      accumulate, launch_info(h, s)) ? SFMM_OK : SFMM_ERR_CUDA;
    if (h->dtype == SFMM_F64)
        return launch_batch<double>(h, op, in, out, shift, p_in, p_out, count, accumulate, s, h->t64);
    return launch_batch<float>(h, op, in, out, shift, p_in, p_out, count, accumulate, s, h->t32);
}

}  // namespace

extern "C" {

const char *sfmm_status_string(sfmm_status s) {
    switch (s) {
        case SFMM_OK: return "SFMM_OK";
        case SFMM_ERR_ARG: return "SFMM_ERR_ARG: invalid argument";
        case SFMM_ERR_ORDER: return "SFMM_ERR_ORDER: expansion order out of range";
        case SFMM_ERR_NOMEM: return "SFMM_ERR_NOMEM: allocation failed";
        case SFMM_ERR_CUDA: return "SFMM_ERR_CUDA: CUDA runtime error";
        case SFMM_ERR_TIMEOUT: return "SFMM_ERR_TIMEOUT: bounded device wait gave up";
        case SFMM_ERR_UNSUPPORTED: return "SFMM_ERR_UNSUPPORTED: request not supported by this build";
        case SFMM_ERR_DEVICE: return "SFMM_ERR_DEVICE: a kernel reported invalid input";
    }
    return "SFMM_ERR_?: unknown status";
}

sfmm_status sfmm_create(int P_max, sfmm_dtype dtype, sfmm_handle *out) {
    SfmmRange nvtx_range("sfmm_create");
    if (out == nullptr) return SFMM_ERR_ARG;
    *out = nullptr;
    if (dtype != SFMM_F64 && dtype != SFMM_F32) return SFMM_ERR_ARG;
    const int lim = dtype == SFMM_F64 ? kMaxPmax64 : kMaxPmax32;
    if (P_max < 1 || P_max > lim) return SFMM_ERR_ORDER;
    sfmm_ctx *h = new (std::nothrow) sfmm_ctx;
    if (h == nullptr) return SFMM_ERR_NOMEM;
    h->Pmax = P_max;
    h->dtype = dtype;
    int dev = 0, smc = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&smc, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
        delete h;
        return SFMM_ERR_CUDA;
    }
    h->device = dev;
    h->sm_count = smc;
    h->smem_optin = (size_t)optin;
    HostTables ht;
    try {
        if (build_tables(P_max, &ht) != 0) { delete h; return SFMM_ERR_ORDER; }
    } catch (...) {
        delete h;
        return SFMM_ERR_NOMEM;
    }
    sfmm_status st = dtype == SFMM_F64 ? upload<double>(ht, h, &h->t64) : upload<float>(ht, h, &h->t32);
    if (st == SFMM_OK && cudaMalloc(&h->d_status, sizeof(int)) != cudaSuccess) st = SFMM_ERR_NOMEM;
    if (st == SFMM_OK && cudaMalloc(&h->d_work, sizeof(unsigned long long)) != cudaSuccess) st = SFMM_ERR_NOMEM;
    if (st == SFMM_OK && cudaMalloc(&h->d_pass, 2 * MAX_PASS_PHASES * sizeof(unsigned long long)) != cudaSuccess)
        st = SFMM_ERR_NOMEM;
    if (st == SFMM_OK && cudaMemset(h->d_status, 0, sizeof(int)) != cudaSuccess) st = SFMM_ERR_CUDA;
    if (st == SFMM_OK) {
        const size_t esz = dtype == SFMM_F64 ? sizeof(double) : sizeof(float);
        {
            // eight resident warps per SM (two per sub-partition); a lane's slot
            // holds a rotated solid and an output solid of order P_max (the
            // group-lists kernels use both)
            h->scratch_bytes = (size_t)smc * 8 * WARP * 2 * x_elems(P_max) * esz;
            if (cudaMalloc(&h->d_scratch, h->scratch_bytes) != cudaSuccess) st = SFMM_ERR_NOMEM;
            else if (cudaEventCreateWithFlags(&h->scratch_free, cudaEventDisableTiming) != cudaSuccess)
                st = SFMM_ERR_CUDA;
        }
    }
    if (st == SFMM_OK) {
        st = fill_unrolled_constants(dev, h->smem_optin);
        h->unrolled_ok = (st == SFMM_OK);
    }
    if (st == SFMM_OK) {
        if (dtype == SFMM_F64) set_kernel_attrs<double>(h->smem_optin);
        else set_kernel_attrs<float>(h->smem_optin);
        if (cudaGetLastError() != cudaSuccess) st = SFMM_ERR_CUDA;
    }
    if (st != SFMM_OK) {
        cudaFree(h->d_tables);
        cudaFree(h->d_status);
        cudaFree(h->d_work);
        cudaFree(h->d_pass);
        cudaFree(h->d_scratch);
        if (h->scratch_free) cudaEventDestroy(h->scratch_free);
        delete h;
        return st;
    }
    *out = h;
    return SFMM_OK;
}

sfmm_status sfmm_destroy(sfmm_handle h) {
    if (h == nullptr) return SFMM_OK;
    cudaDeviceSynchronize();
    cudaFree(h->d_tables);
    cudaFree(h->d_status);
    cudaFree(h->d_work);
    cudaFree(h->d_pass);
    cudaFree(h->d_scratch);
    if (h->scratch_free) cudaEventDestroy(h->scratch_free);
    delete h;
    return SFMM_OK;
}

sfmm_status sfmm_get_info(sfmm_handle h, int *P_max, sfmm_dtype *dtype) {
    if (h == nullptr) return SFMM_ERR_ARG;
    if (P_max) *P_max = h->Pmax;
    if (dtype) *dtype = h->dtype;
    return SFMM_OK;
}

sfmm_status sfmm_m2m_batch(sfmm_handle h, const void *const *in, void *const *out,
                           const void *shift, int p_in, int p_out, long long count,
                           int accumulate, sfmm_stream stream) {
    SfmmRange nvtx_range("sfmm_m2m_batch");
    return batch(h, OP_M2M, in, out, shift, p_in, p_out, count, accumulate, stream);
}

sfmm_status sfmm_m2l_batch(sfmm_handle h, const void *const *in, void *const *out,
                           const void *shift, int p_in, int p_out, long long count,
                           int accumulate, sfmm_stream stream) {
    SfmmRange nvtx_range("sfmm_m2l_batch");
    return batch(h, OP_M2L, in, out, shift, p_in, p_out, count, accumulate, stream);
}

sfmm_status sfmm_l2l_batch(sfmm_handle h, const void *const *in, void *const *out,
                           const void *shift, int p_in, int p_out, long long count,
                           int accumulate, sfmm_stream stream) {
    SfmmRange nvtx_range("sfmm_l2l_batch");
    return batch(h, OP_L2L, in, out, shift, p_in, p_out, count, accumulate, stream);
}

sfmm_status sfmm_translate_lists(sfmm_handle h, sfmm_op op, const void *const *src,
                                 const void *shift, const long long *offsets,
                                 void *const *out, int p_in, int p_out,
                                 long long n_targets, int accumulate, sfmm_stream stream) {
    SfmmRange nvtx_range("sfmm_translate_lists");
    sfmm_status st = check_common(h, p_in, p_out, n_targets);
    if (st != SFMM_OK) return st;
    if (op != SFMM_M2M && op != SFMM_M2L && op != SFMM_L2L) return SFMM_ERR_ARG;
    if (n_targets == 0) return SFMM_OK;
    if (src == nullptr || shift == nullptr || offsets == nullptr || out == nullptr) return SFMM_ERR_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (use_unrolled(h, (int)op, p_in, p_out))
        return unrolled::launch_lists(h->dtype == SFMM_F64, p_in, (int)op, src, shift, offsets, out,
                                      n_targets, accumulate, launch_info(h, s)) ? SFMM_OK : SFMM_ERR_CUDA;
    if (h->dtype == SFMM_F64)
        return launch_lists<double>(h, (int)op, src, shift, offsets, out, p_in, p_out, n_targets, accumulate, s, h->t64);
    return launch_lists<float>(h, (int)op, src, shift, offsets, out, p_in, p_out, n_targets, accumulate, s, h->t32);
}

static sfmm_status p2x(sfmm_handle h, bool singular, int P, const void *points, const void *q,
                       const long long *offsets, const void *centres, void *out,
                       long long n_boxes, sfmm_stream stream) {
    sfmm_status st = check_common(h, P, P, n_boxes);
    if (st != SFMM_OK) return st;
    if (n_boxes == 0) return SFMM_OK;
    if (points == nullptr || q == nullptr || offsets == nullptr || centres == nullptr || out == nullptr)
        return SFMM_ERR_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (h->dtype == SFMM_F64)
        return launch_p2x<double>(h, singular, P, points, q, offsets, centres, out, n_boxes, s);
    return launch_p2x<float>(h, singular, P, points, q, offsets, centres, out, n_boxes, s);
}

sfmm_status sfmm_p2m_boxes(sfmm_handle h, int P, const void *points, const void *q,
                           const long long *offsets, const void *centres, void *out,
                           long long n_boxes, sfmm_stream stream) {
    SfmmRange nvtx_range("sfmm_p2m_boxes");
    return p2x(h, false, P, points, q, offsets, centres, out, n_boxes, stream);
}

sfmm_status sfmm_p2l_boxes(sfmm_handle h, int P, const void *points, const void *q,
                           const long long *offsets, const void *centres, void *out,
                           long long n_boxes, sfmm_stream stream) {
    SfmmRange nvtx_range("sfmm_p2l_boxes");
    return p2x(h, true, P, points, q, offsets, centres, out, n_boxes, stream);
}

sfmm_status sfmm_sync_status(sfmm_handle h, sfmm_stream stream, int *device_status) {
    if (h == nullptr) return SFMM_ERR_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int v = 0;
    if (cudaMemcpyAsync(&v, h->d_status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return SFMM_ERR_CUDA;
    if (v != 0 && cudaMemsetAsync(h->d_status, 0, sizeof(int), s) != cudaSuccess) return SFMM_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return SFMM_ERR_CUDA;
    if (device_status) *device_status = v;
    return v == 0 ? SFMM_OK : SFMM_ERR_DEVICE;
}

sfmm_status sfmm_set_policy(sfmm_handle h, sfmm_op op, int p_in, int p_out, sfmm_policy policy,
                            int warps_per_block) {
    if (h == nullptr || (op != SFMM_M2M && op != SFMM_M2L && op != SFMM_L2L)) return SFMM_ERR_ARG;
    if (policy < SFMM_POLICY_AUTO || policy > SFMM_POLICY_WIDE || warps_per_block < 0 ||
        warps_per_block > 8)
        return SFMM_ERR_ARG;
    if (p_in < 1 || p_out < 1 || p_in > h->Pmax || p_out > h->Pmax) return SFMM_ERR_ORDER;
    const size_t sz = h->dtype == SFMM_F64 ? sizeof(double) : sizeof(float);
    if (policy == SFMM_POLICY_UNROLLED && !(p_in == p_out && unrolled::compiled(p_in) && h->unrolled_ok))
        return SFMM_ERR_UNSUPPORTED;
    if (policy == SFMM_POLICY_SHARED &&
        (size_t)(x_elems(p_in) + row_elems(p_in, p_out)) * WARP * sz > h->smem_optin)
        return SFMM_ERR_UNSUPPORTED;
    if (policy == SFMM_POLICY_GLOBAL &&
        (h->d_scratch == nullptr || (size_t)x_elems(p_in) * WARP * sz > h->scratch_bytes))
        return SFMM_ERR_UNSUPPORTED;
    if (policy == SFMM_POLICY_WIDE &&
        ((p_in > p_out ? p_in : p_out) > wide_max_order() ||
         (size_t)wide_warp_bytes(p_in > p_out ? p_in : p_out) * (warps_per_block > 0 ? warps_per_block : 1) >
             h->smem_optin))
        return SFMM_ERR_UNSUPPORTED;
    h->policy[op][p_in][p_out] = (unsigned char)policy;
    h->warps[op][p_in][p_out] = (unsigned char)warps_per_block;
    return SFMM_OK;
}

sfmm_status sfmm_reserve_scratch(sfmm_handle h, int p_in_max) {
    if (h == nullptr) return SFMM_ERR_ARG;
    if (p_in_max < 1 || p_in_max > h->Pmax) return SFMM_ERR_ORDER;
    const size_t sz = h->dtype == SFMM_F64 ? sizeof(double) : sizeof(float);
    const size_t need = (size_t)h->sm_count * 8 * WARP * 2 * x_elems(p_in_max) * sz;
    std::lock_guard<std::mutex> lk(h->scratch_mu);
    if (h->d_scratch != nullptr && h->scratch_bytes >= need) return SFMM_OK;
    if (cudaDeviceSynchronize() != cudaSuccess) return SFMM_ERR_CUDA;
    void *p = nullptr;
    if (cudaMalloc(&p, need) != cudaSuccess) return SFMM_ERR_NOMEM;
    if (h->scratch_free == nullptr &&
        cudaEventCreateWithFlags(&h->scratch_free, cudaEventDisableTiming) != cudaSuccess) {
        cudaFree(p);
        return SFMM_ERR_CUDA;
    }
    cudaFree(h->d_scratch);
    h->d_scratch = p;
    h->scratch_bytes = need;
    return SFMM_OK;
}

}  // extern "C"

template <typename T>
static sfmm_status launch_multi(sfmm_handle h, const sfmm_list_class *classes, int n,
                                const void *const *src, const void *shift,
                                const long long *offsets, void *const *out, int accumulate,
                                cudaStream_t stream, const DevTables<T> &tb) {
    MultiParams mp{};
    mp.n = n;
    int xs = 0, rs = 0;
    long long chunks = 0;
    for (int k = 0; k < n; ++k) {
        const sfmm_list_class &c = classes[k];
        MultiClass &m = mp.c[k];
        m.op = c.op;
        m.p_in = c.p_in;
        m.p_out = c.p_out;
        m.g = c.lanes_per_target > 0 ? c.lanes_per_target : default_lanes(c.op);
        m.tb = c.target_begin;
        m.te = c.target_end;
        m.chunk_begin = chunks;
        const int per_chunk = WARP / m.g;
        chunks += (c.target_end - c.target_begin + per_chunk - 1) / per_chunk;
        const int xk = x_elems(c.p_in) + (m.g > 1 ? c.p_out * (c.p_out + 1) : 0);
        xs = xs > xk ? xs : xk;
        rs = rs > row_elems(c.p_in, c.p_out) ? rs : row_elems(c.p_in, c.p_out);
    }
    mp.total_chunks = chunks;
    mp.x_slot = xs;
    mp.row_slot = rs;
    if (chunks == 0) return SFMM_OK;
    const size_t per_warp = (size_t)rs * WARP * sizeof(T);
    const size_t slot = (size_t)xs * WARP * sizeof(T);
    if (h->d_scratch == nullptr || per_warp > h->smem_optin || slot > h->scratch_bytes)
        return SFMM_ERR_UNSUPPORTED;
    int w = (int)(h->smem_optin / 2 / per_warp);
    if (w < 1) w = 1;
    if (w > 4) w = 4;
    long long slots = (long long)(h->scratch_bytes / slot);
    if (w > slots) w = (int)slots;
    long long blocks = slots / w;
    const long long need = (chunks + w - 1) / w;
    if (blocks > need) blocks = need;
    if (blocks > 0x7fffffffLL) blocks = 0x7fffffffLL;
    Geometry g;
    g.xg = true;
    g.warps = w;
    g.smem = (size_t)w * per_warp;
    g.blocks = blocks;
    ScratchGuard guard(h, stream, true);
    mp.work = h->d_work;                          // chunks are handed out by this counter
    if (cudaMemsetAsync(h->d_work, 0, sizeof(unsigned long long), stream) != cudaSuccess) return SFMM_ERR_CUDA;
    multi_launch<T>(h, g, stream, tb, mp, reinterpret_cast<const T *const *>(src), reinterpret_cast<const T *>(shift),
                    offsets, reinterpret_cast<T *const *>(out), accumulate, reinterpret_cast<T *>(h->d_scratch),
                    h->d_status);
    return cudaGetLastError() == cudaSuccess ? SFMM_OK : SFMM_ERR_CUDA;
}

// One launch for a whole pass: classes grouped into phases (sfmm_translate_pass).
template <typename T>
static sfmm_status launch_pass(sfmm_handle h, const sfmm_pass_class *classes, int n, cudaStream_t stream,
                               const DevTables<T> &tb) {
    std::unique_ptr<PassParams> pp(new (std::nothrow) PassParams());
    if (!pp) return SFMM_ERR_NOMEM;
    int xs = 0, rs = 0, nph = 0;
    long long chunks = 0;
    for (int k = 0; k < n; ++k) {
        const sfmm_pass_class &c = classes[k];
        if (k == 0 || c.phase != classes[k - 1].phase) {
            if (nph == MAX_PASS_PHASES) return SFMM_ERR_UNSUPPORTED;
            if (nph > 0) {
                pp->ph[nph - 1].chunk_end = chunks;
                pp->ph[nph - 1].class_end = k;
            }
            pp->ph[nph].chunk_begin = chunks;
            pp->ph[nph].class_begin = k;
            ++nph;
        }
        PassClass &m = pp->c[k];
        m.src = static_cast<const void *>(c.src);
        m.shift = c.shift;
        m.offsets = c.offsets;
        m.out = static_cast<void *>(const_cast<void **>(c.out));
        m.n_targets = c.n_targets;
        m.op = c.op;
        m.p_in = c.p_in;
        m.p_out = c.p_out;
        m.g = c.lanes_per_target > 0 ? c.lanes_per_target : default_lanes(c.op);
        m.accumulate = c.accumulate != 0;
        m.chunk_begin = chunks;
        const int per_chunk = WARP / m.g;
        chunks += (c.n_targets + per_chunk - 1) / per_chunk;
        const int xk = x_elems(c.p_in) + (m.g > 1 ? c.p_out * (c.p_out + 1) : 0);
        xs = xs > xk ? xs : xk;
        rs = rs > row_elems(c.p_in, c.p_out) ? rs : row_elems(c.p_in, c.p_out);
    }
    pp->ph[nph - 1].chunk_end = chunks;
    pp->ph[nph - 1].class_end = n;
    pp->n_phases = nph;
    pp->x_slot = xs;
    pp->row_slot = rs;
    const size_t per_warp = (size_t)rs * WARP * sizeof(T);
    const size_t slot = (size_t)xs * WARP * sizeof(T);
    if (h->d_scratch == nullptr || per_warp > h->smem_optin || slot > h->scratch_bytes)
        return SFMM_ERR_UNSUPPORTED;
    int w = (int)(h->smem_optin / 2 / per_warp);
    if (w < 1) w = 1;
    if (w > 4) w = 4;
    const long long slots = (long long)(h->scratch_bytes / slot);
    if (w > slots) w = (int)slots;
    Geometry g;
    g.xg = true;
    g.warps = w;
    g.smem = (size_t)w * per_warp;
    long long blocks = slots / w;
    const long long resident = pass_resident_blocks<T>(h, g);
    if (resident < 0) return SFMM_ERR_CUDA;
    if (blocks > resident) blocks = resident;
    if (blocks < 1) return SFMM_ERR_UNSUPPORTED;
    g.blocks = blocks;
    ScratchGuard guard(h, stream, true);
    if (cudaMemsetAsync(h->d_pass, 0, 2 * MAX_PASS_PHASES * sizeof(unsigned long long), stream) != cudaSuccess)
        return SFMM_ERR_CUDA;
    if (pass_launch<T>(h, g, stream, tb, *pp, reinterpret_cast<T *>(h->d_scratch), h->d_pass, h->d_status) != cudaSuccess)
        return SFMM_ERR_CUDA;
    return cudaGetLastError() == cudaSuccess ? SFMM_OK : SFMM_ERR_CUDA;
}

extern "C" {

sfmm_status sfmm_translate_pass(sfmm_handle h, const sfmm_pass_class *classes, int n_classes,
                                sfmm_stream stream) {
    SfmmRange nvtx_range("sfmm_translate_pass");
    if (h == nullptr || classes == nullptr || n_classes < 1 || n_classes > SFMM_MAX_PASS_CLASSES)
        return SFMM_ERR_ARG;
    for (int k = 0; k < n_classes; ++k) {
        const sfmm_pass_class &c = classes[k];
        if (c.op != SFMM_M2M && c.op != SFMM_M2L && c.op != SFMM_L2L) return SFMM_ERR_ARG;
        if (c.n_targets < 0 || (k > 0 && c.phase < classes[k - 1].phase)) return SFMM_ERR_ARG;
        const int g = c.lanes_per_target;
        if (g != 0 && g != 1 && g != 2 && g != 4 && g != 8 && g != 16 && g != 32) return SFMM_ERR_ARG;
        if (c.p_in < 1 || c.p_out < 1 || c.p_in > h->Pmax || c.p_out > h->Pmax) return SFMM_ERR_ORDER;
        if (c.n_targets > 0 && (c.src == nullptr || c.shift == nullptr || c.offsets == nullptr || c.out == nullptr))
            return SFMM_ERR_ARG;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (h->dtype == SFMM_F64) return launch_pass<double>(h, classes, n_classes, s, h->t64);
    return launch_pass<float>(h, classes, n_classes, s, h->t32);
}

}  // extern "C"

extern "C" {

sfmm_status sfmm_translate_lists_multi(sfmm_handle h, const sfmm_list_class *classes,
                                       int n_classes, const void *const *src,
                                       const void *shift, const long long *offsets,
                                       void *const *out, int accumulate, sfmm_stream stream) {
    SfmmRange nvtx_range("sfmm_translate_lists_multi");
    if (h == nullptr || classes == nullptr || n_classes < 1 || n_classes > SFMM_MAX_CLASSES)
        return SFMM_ERR_ARG;
    for (int k = 0; k < n_classes; ++k) {
        const sfmm_list_class &c = classes[k];
        if (c.op != SFMM_M2M && c.op != SFMM_M2L && c.op != SFMM_L2L) return SFMM_ERR_ARG;
        if (c.target_begin < 0 || c.target_end < c.target_begin) return SFMM_ERR_ARG;
        const int g = c.lanes_per_target;
        if (g != 0 && g != 1 && g != 2 && g != 4 && g != 8 && g != 16 && g != 32) return SFMM_ERR_ARG;
        if (c.p_in < 1 || c.p_out < 1 || c.p_in > h->Pmax || c.p_out > h->Pmax) return SFMM_ERR_ORDER;
    }
    if (src == nullptr || shift == nullptr || offsets == nullptr || out == nullptr) return SFMM_ERR_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (h->dtype == SFMM_F64)
        return launch_multi<double>(h, classes, n_classes, src, shift, offsets, out, accumulate, s, h->t64);
    return launch_multi<float>(h, classes, n_classes, src, shift, offsets, out, accumulate, s, h->t32);
}

sfmm_status sfmm_host_swap_matrices(int n, double *F, double *G) {
    if (F == nullptr || G == nullptr) return SFMM_ERR_ARG;
    if (n < 0 || n > 63) return SFMM_ERR_ORDER;
    return dense_swap_matrices(n, F, G) == 0 ? SFMM_OK : SFMM_ERR_ORDER;
}

sfmm_status sfmm_host_ztranslate(sfmm_op op, int P, int m, double *T) {
    if (T == nullptr || (op != SFMM_M2M && op != SFMM_M2L && op != SFMM_L2L)) return SFMM_ERR_ARG;
    if (P < 1 || P > 64 || m < 0 || m >= P) return SFMM_ERR_ORDER;
    HostTables ht;
    if (build_tables(P, &ht) != 0) return SFMM_ERR_ORDER;
    const long long base = ztrans_block_offset(P, m);
    const size_t n = (size_t)(P - m) * (P - m);
    std::memcpy(T, ht.Tz[op].data() + base, n * sizeof(double));
    return SFMM_OK;
}

}  // extern "C"
