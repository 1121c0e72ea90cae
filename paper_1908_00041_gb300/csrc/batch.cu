// Ragged batches (fields of different degree L in one call) and the generator autotuner.
//
// A batch plan groups its fields by degree; each group is an ordinary plan whose user-
// buffer kernels (longitude DFTs, combine, uncombine, polar patch) address the fields of
// that degree inside the caller's packed buffers through per-field offset tables.  For
// the split-precision form the tensor-core Legendre stage of all groups runs as ONE
// persistent launch: the work items of every group are merged into one longest-first
// queue, each item naming its group's operand tensor maps and output buffer.  The whole
// call can be replayed as a CUDA graph (captured on the second call with the same
// buffers).
//
// Autotuner: the FP64 recurrence generator runs 128 threads per block arranged as
// (128 / lt) orders x lt latitudes, each block covering mb such order groups.  For every
// degree the tuner times the candidate (lt, mb) shapes on the device and keeps the
// fastest; small degrees (few latitudes) favour narrow latitude tiles and several
// orders per block, large ones wide tiles.
#include <algorithm>
#include <map>
#include <new>
#include <vector>

#include "favest_internal.h"

using namespace favest;

namespace {

struct GraphCache {
    const void *ptr[4] = {nullptr, nullptr, nullptr, nullptr};
    int seen = 0;                     // calls made with these buffers
    cudaGraphExec_t exec = nullptr;
};

}  // namespace

struct favest_batch_s {
    int nfields = 0, precision = 0, io = 0, flags = 0;
    std::vector<int> L;                       // per field
    std::vector<long long> toff, coff;        // per field (elements)
    long long field_elems = 0, coef_elems = 0;
    std::vector<favest_plan> groups;          // one plan per distinct degree (ascending)
    std::vector<int> group_L, group_n;
    std::vector<long long *> d_toff, d_coff;  // per group, device
    GemmGroup *d_gg = nullptr;                // [2 * groups]: forward, adjoint of each group
    TcItem *d_items_f = nullptr, *d_items_a = nullptr;
    int n_items_f = 0, n_items_a = 0;
    int *d_status = nullptr;
    int num_sms = 0, device = 0;
    cudaStream_t cap = nullptr;               // capture stream
    GraphCache graph[2];                      // forward, adjoint
    // one stream per degree group for the per-group kernels, forked from and joined back
    // into the call's stream around the merged tensor-core launch (parallel branches of
    // the captured graph)
    std::vector<cudaStream_t> gstream;
    std::vector<cudaEvent_t> gjoin;
    cudaEvent_t fork = nullptr;
};

namespace {

bool same_ptrs(const GraphCache &g, const void *const p[4])
{
    for (int i = 0; i < 4; ++i)
        if (g.ptr[i] != p[i]) return false;
    return true;
}

template <typename T>
cudaError_t upload_vec(T **d, const std::vector<T> &h)
{
    if (h.empty()) return cudaSuccess;
    cudaError_t e = plan_malloc((void **)d, h.size() * sizeof(T));
    if (e != cudaSuccess) return e;
    return cudaMemcpy(*d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
}

// Runs fn(g, stream) for every degree group on the group's own stream, largest degree
// first, after all work queued so far on s, and makes s wait for all of them.
template <typename Fn>
cudaError_t per_group(favest_batch_s &bp, cudaStream_t s, Fn fn)
{
    const int G = (int)bp.groups.size();
    cudaError_t e = cudaEventRecord(bp.fork, s);
    for (int g = G - 1; g >= 0 && e == cudaSuccess; --g) {
        e = cudaStreamWaitEvent(bp.gstream[g], bp.fork, 0);
        if (e == cudaSuccess) e = fn(g, bp.gstream[g]);
        if (e == cudaSuccess) e = cudaEventRecord(bp.gjoin[g], bp.gstream[g]);
    }
    for (int g = 0; g < G && e == cudaSuccess; ++g) e = cudaStreamWaitEvent(s, bp.gjoin[g], 0);
    return e;
}

// The launch sequence of one batched transform on stream s.
cudaError_t enqueue(favest_batch_s &bp, bool adjoint, const void *Tth, const void *Tph, const void *a,
                    const void *b, cudaStream_t s)
{
    cudaError_t e = cudaSuccess;
    if (bp.precision != FAVEST_BF16X6) {
        // no shared stage: each group's whole transform is one branch
        return per_group(bp, s, [&](int g, cudaStream_t gs) {
            int st = adjoint ? favest_adj(bp.groups[g], a, b, (void *)Tth, (void *)Tph, gs)
                             : favest_fwd(bp.groups[g], Tth, Tph, (void *)a, (void *)b, gs);
            return st == FAVEST_OK ? cudaSuccess : cudaErrorLaunchFailure;
        });
    }
    if (!adjoint) {
        e = per_group(bp, s, [&](int g, cudaStream_t gs) {
            const Plan &p = bp.groups[g]->p;
            cudaError_t r = launch_fft_fwd_bf16(p, Tth, Tph, gs);
            return r == cudaSuccess ? launch_gen_lambda(p, kGenFwd, gs) : r;
        });
        if (e == cudaSuccess)
            e = launch_tc_gemm_items(256, bp.d_gg, bp.d_items_f, bp.n_items_f, 1, bp.d_status, bp.num_sms, s);
        if (e == cudaSuccess)
            e = per_group(bp, s, [&](int g, cudaStream_t gs) {
                return launch_combine_bf16(bp.groups[g]->p, (void *)a, (void *)b, gs);
            });
    } else {
        e = per_group(bp, s, [&](int g, cudaStream_t gs) {
            const Plan &p = bp.groups[g]->p;
            cudaError_t r = launch_uncombine_bf16(p, a, b, gs);
            return r == cudaSuccess ? launch_gen_lambda(p, kGenAdj, gs) : r;
        });
        if (e == cudaSuccess)
            e = launch_tc_gemm_items(256, bp.d_gg, bp.d_items_a, bp.n_items_a, 0, bp.d_status, bp.num_sms, s);
        if (e == cudaSuccess)
            e = per_group(bp, s, [&](int g, cudaStream_t gs) {
                const Plan &p = bp.groups[g]->p;
                cudaError_t r = p.pol_jc > 0 ? launch_polar_patch(p, a, b, gs) : cudaSuccess;
                return r == cudaSuccess ? launch_fft_inv_bf16(p, (void *)Tth, (void *)Tph, gs) : r;
            });
    }
    return e;
}

int run_batched(favest_batch bp, bool adjoint, const void *Tth, const void *Tph, const void *a, const void *b,
                void *stream)
{
    if (!bp || !Tth || !Tph || !a || !b) return FAVEST_EINVAL;
    const size_t al = (bp->precision == FAVEST_BF16X6 || bp->io != FAVEST_IO_C64) ? 16 : 8;
    if ((((uintptr_t)Tth | (uintptr_t)Tph) % al) || (((uintptr_t)a | (uintptr_t)b) % 8)) return FAVEST_EINVAL;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != bp->device) return FAVEST_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const void *ptrs[4] = {Tth, Tph, a, b};
    GraphCache &gc = bp->graph[adjoint ? 1 : 0];
    if (!(bp->flags & FAVEST_BATCH_GRAPH)) {
        return enqueue(*bp, adjoint, Tth, Tph, a, b, s) == cudaSuccess ? FAVEST_OK : FAVEST_ECUDA;
    }
    if (gc.exec && same_ptrs(gc, ptrs))
        return cudaGraphLaunch(gc.exec, s) == cudaSuccess ? FAVEST_OK : FAVEST_ECUDA;
    if (!same_ptrs(gc, ptrs) || gc.seen == 0) {
        // first call with these buffers: run eagerly (this also configures every kernel)
        if (gc.exec) {
            cudaGraphExecDestroy(gc.exec);
            gc.exec = nullptr;
        }
        for (int i = 0; i < 4; ++i) gc.ptr[i] = ptrs[i];
        gc.seen = 1;
        return enqueue(*bp, adjoint, Tth, Tph, a, b, s) == cudaSuccess ? FAVEST_OK : FAVEST_ECUDA;
    }
    // second call with the same buffers: capture the sequence once, then replay it
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(bp->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return FAVEST_ECUDA;
    cudaError_t e = enqueue(*bp, adjoint, Tth, Tph, a, b, bp->cap);
    cudaError_t e2 = cudaStreamEndCapture(bp->cap, &graph);
    if (e != cudaSuccess || e2 != cudaSuccess || !graph) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return FAVEST_ECUDA;
    }
    e = cudaGraphInstantiate(&gc.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        gc.exec = nullptr;
        return FAVEST_ECUDA;
    }
    return cudaGraphLaunch(gc.exec, s) == cudaSuccess ? FAVEST_OK : FAVEST_ECUDA;
}

void destroy_batch(favest_batch_s *bp)
{
    cudaDeviceSynchronize();
    for (auto &g : bp->graph)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    for (auto p : bp->groups) favest_plan_destroy(p);
    for (auto d : bp->d_toff)
        if (d) cudaFree(d);
    for (auto d : bp->d_coff)
        if (d) cudaFree(d);
    void *ptrs[] = {bp->d_gg, bp->d_items_f, bp->d_items_a, bp->d_status};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    if (bp->cap) cudaStreamDestroy(bp->cap);
    for (auto q : bp->gstream)
        if (q) cudaStreamDestroy(q);
    for (auto ev : bp->gjoin)
        if (ev) cudaEventDestroy(ev);
    if (bp->fork) cudaEventDestroy(bp->fork);
    delete bp;
}

// Generator shapes the tuner times and favest_plan_set_gen_shape accepts:
// (latitudes per block, order groups per block, latitude chains per thread)
constexpr int kGenShapes[][3] = {{128, 1, 2}, {64, 1, 2}, {32, 1, 2}, {128, 2, 2}, {64, 2, 2}, {32, 2, 2},
                                 {32, 4, 2},  {128, 1, 1}, {64, 1, 1}, {32, 1, 1}, {128, 2, 1}, {64, 2, 1},
                                 {32, 2, 1},  {32, 4, 1}};

}  // namespace

extern "C" {

int favest_plan_set_gen_shape(favest_plan plan, int lt, int mb, int nj)
{
    if (!plan) return FAVEST_EINVAL;
    bool known = false;
    for (const auto &c : kGenShapes) known = known || (c[0] == lt && c[1] == mb && c[2] == nj);
    if (!known) return FAVEST_EINVAL;
    Plan &p = plan->p;
    if (p.precision != FAVEST_BF16X6) return FAVEST_OK;   // no generator on the FP64 path
    p.gen_lt = lt;
    p.gen_mb = mb;
    p.gen_nj = nj;
    return FAVEST_OK;
}

int favest_plan_tune(favest_plan plan, void *stream)
{
    if (!plan) return FAVEST_EINVAL;
    Plan &p = plan->p;
    if (p.precision != FAVEST_BF16X6) return FAVEST_OK;   // nothing tunable on the FP64 path
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return FAVEST_ECUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return FAVEST_ECUDA;
    }
    float best = 1e30f;
    int blt = p.gen_lt, bmb = p.gen_mb, bnj = p.gen_nj, st = FAVEST_OK;
    for (const auto &c : kGenShapes) {
        if (launch_gen_lambda_shape(p, kGenFwd, c[0], c[1], c[2], s) != cudaSuccess) {
            st = FAVEST_ECUDA;
            break;
        }
        cudaEventRecord(e0, s);
        for (int r = 0; r < 3; ++r) launch_gen_lambda_shape(p, kGenFwd, c[0], c[1], c[2], s);
        cudaEventRecord(e1, s);
        float ms = 0.f;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            st = FAVEST_ECUDA;
            break;
        }
        if (ms < best) {
            best = ms;
            blt = c[0];
            bmb = c[1];
            bnj = c[2];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st == FAVEST_OK) {
        p.gen_lt = blt;
        p.gen_mb = bmb;
        p.gen_nj = bnj;
    }
    return st;
}

int favest_plan_gen_chains(favest_plan plan) { return plan ? plan->p.gen_nj : FAVEST_EINVAL; }

int favest_plan_gen_shape(favest_plan plan, int *lt, int *mb)
{
    if (!plan || !lt || !mb) return FAVEST_EINVAL;
    *lt = plan->p.gen_lt;
    *mb = plan->p.gen_mb;
    return FAVEST_OK;
}

int favest_batch_create(int nfields, const int *L, const long long *field_off, const long long *coef_off,
                        int precision, int io_type, int flags, favest_batch *out)
{
    if (!out) return FAVEST_EINVAL;
    *out = nullptr;
    if (nfields < 1 || !L) return FAVEST_EINVAL;
    if (precision != FAVEST_FP64 && precision != FAVEST_BF16X6) return FAVEST_EINVAL;
    if (io_type != FAVEST_IO_C128 && io_type != FAVEST_IO_C64 && io_type != FAVEST_IO_R32 &&
        io_type != FAVEST_IO_R64)
        return FAVEST_EINVAL;
    const bool real = io_type == FAVEST_IO_R32 || io_type == FAVEST_IO_R64;
    // field planes start on 16 bytes: offsets in elements of the io type
    const long long align = io_type == FAVEST_IO_R32 ? 4 : (io_type == FAVEST_IO_C128 ? 1 : 2);
    if (flags & ~(FAVEST_BATCH_AUTOTUNE | FAVEST_BATCH_GRAPH)) return FAVEST_EINVAL;
    for (int i = 0; i < nfields; ++i)
        if (L[i] < 1) return FAVEST_EINVAL;
    favest_batch_s *bp = new (std::nothrow) favest_batch_s();
    if (!bp) return FAVEST_ENOMEM;
    bp->nfields = nfields;
    bp->precision = precision;
    bp->io = io_type;
    bp->flags = flags;
    bp->L.assign(L, L + nfields);
    bp->toff.resize(nfields);
    bp->coff.resize(nfields);
    long long fo = 0, co = 0;
    for (int i = 0; i < nfields; ++i) {
        const long long fe = (long long)(L[i] + 1) * 2 * (L[i] + 1);
        const long long ce = real ? (long long)L[i] * (L[i] + 3) / 2 : (long long)L[i] * L[i] + 2LL * L[i];
        bp->toff[i] = field_off ? field_off[i] : fo;
        bp->coff[i] = coef_off ? coef_off[i] : co;
        if (bp->toff[i] < 0 || bp->coff[i] < 0 || (bp->toff[i] % align)) {
            delete bp;
            return FAVEST_EINVAL;   // field planes must start on 16 bytes
        }
        bp->field_elems = std::max(bp->field_elems, bp->toff[i] + fe);
        bp->coef_elems = std::max(bp->coef_elems, bp->coff[i] + ce);
        fo += (fe + align - 1) / align * align;   // default packing keeps planes on 16 bytes
        co += ce;
    }
    if (cudaGetDevice(&bp->device) != cudaSuccess) {
        delete bp;
        return FAVEST_ECUDA;
    }
    cudaDeviceGetAttribute(&bp->num_sms, cudaDevAttrMultiProcessorCount, bp->device);
    // groups by degree
    std::map<int, std::vector<int>> byL;
    for (int i = 0; i < nfields; ++i) byL[L[i]].push_back(i);
    int st = FAVEST_OK;
    std::vector<GemmGroup> gg;
    std::vector<TcItem> itf, ita;
    for (auto &kv : byL) {
        favest_plan gp = nullptr;
        st = plan_create_internal(kv.first, (int)kv.second.size(), precision, io_type, nullptr, nullptr,
                                  precision == FAVEST_BF16X6 ? 256 : 0, &gp);
        if (st != FAVEST_OK) break;
        bp->groups.push_back(gp);
        bp->group_L.push_back(kv.first);
        bp->group_n.push_back((int)kv.second.size());
        std::vector<long long> t, c;
        for (int i : kv.second) {
            t.push_back(bp->toff[i]);
            c.push_back(bp->coff[i]);
        }
        long long *dt = nullptr, *dc = nullptr;
        if (upload_vec(&dt, t) != cudaSuccess || upload_vec(&dc, c) != cudaSuccess) {
            if (dt) cudaFree(dt);
            if (dc) cudaFree(dc);
            st = FAVEST_ENOMEM;
            break;
        }
        bp->d_toff.push_back(dt);
        bp->d_coff.push_back(dc);
        gp->p.d_toff = dt;
        gp->p.d_coff = dc;
        if (flags & FAVEST_BATCH_AUTOTUNE) {
            st = favest_plan_tune(gp, nullptr);
            if (st != FAVEST_OK) break;
        }
        if (precision == FAVEST_BF16X6) {
            const Plan &p = gp->p;
            const int g0 = (int)gg.size();
            GemmGroup f, a;
            f.tmap_a = p.tmap_lam_f;
            f.tmap_b = p.tmap_fb;
            f.out = p.d_Q32;
            a.tmap_a = p.tmap_lam_a;
            a.tmap_b = p.tmap_gb;
            a.out = p.d_S32;
            gg.push_back(f);
            gg.push_back(a);
            for (TcItem I : p.h_items_f) {
                I.group = g0;
                itf.push_back(I);
            }
            for (TcItem I : p.h_items_a) {
                I.group = g0 + 1;
                ita.push_back(I);
            }
        }
    }
    if (st == FAVEST_OK && precision == FAVEST_BF16X6) {
        // one queue per direction, heaviest items first
        auto heavier = [](const TcItem &x, const TcItem &y) { return x.nk > y.nk; };
        std::stable_sort(itf.begin(), itf.end(), heavier);
        std::stable_sort(ita.begin(), ita.end(), heavier);
        bp->n_items_f = (int)itf.size();
        bp->n_items_a = (int)ita.size();
        if (upload_vec(&bp->d_gg, gg) != cudaSuccess || upload_vec(&bp->d_items_f, itf) != cudaSuccess ||
            upload_vec(&bp->d_items_a, ita) != cudaSuccess ||
            plan_malloc((void **)&bp->d_status, kStatusWords * sizeof(int)) != cudaSuccess ||
            cudaMemset(bp->d_status, 0, kStatusWords * sizeof(int)) != cudaSuccess)
            st = FAVEST_ENOMEM;
    }
    if (st == FAVEST_OK && cudaStreamCreateWithFlags(&bp->cap, cudaStreamNonBlocking) != cudaSuccess)
        st = FAVEST_ECUDA;
    if (st == FAVEST_OK && cudaEventCreateWithFlags(&bp->fork, cudaEventDisableTiming) != cudaSuccess)
        st = FAVEST_ECUDA;
    for (size_t g = 0; st == FAVEST_OK && g < bp->groups.size(); ++g) {
        cudaStream_t q = nullptr;
        cudaEvent_t ev = nullptr;
        if (cudaStreamCreateWithFlags(&q, cudaStreamNonBlocking) != cudaSuccess) st = FAVEST_ECUDA;
        else bp->gstream.push_back(q);
        if (st == FAVEST_OK && cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) st = FAVEST_ECUDA;
        else if (st == FAVEST_OK) bp->gjoin.push_back(ev);
    }
    if (st == FAVEST_OK && cudaDeviceSynchronize() != cudaSuccess) st = FAVEST_ECUDA;
    if (st != FAVEST_OK) {
        cudaGetLastError();
        destroy_batch(bp);
        return st;
    }
    *out = bp;
    return FAVEST_OK;
}

int favest_fwd_batched(favest_batch batch, const void *Tth, const void *Tph, void *a, void *b, void *stream)
{
    return run_batched(batch, false, Tth, Tph, a, b, stream);
}

int favest_adj_batched(favest_batch batch, const void *a, const void *b, void *Tth, void *Tph, void *stream)
{
    return run_batched(batch, true, Tth, Tph, a, b, stream);
}

int favest_batch_ngroups(favest_batch batch) { return batch ? (int)batch->groups.size() : FAVEST_EINVAL; }

int favest_batch_group(favest_batch batch, int g, int *L, int *nfields, int *gen_lt, int *gen_mb)
{
    if (!batch || g < 0 || g >= (int)batch->groups.size() || !L || !nfields || !gen_lt || !gen_mb)
        return FAVEST_EINVAL;
    *L = batch->group_L[g];
    *nfields = batch->group_n[g];
    *gen_lt = batch->groups[g]->p.gen_lt;
    *gen_mb = batch->groups[g]->p.gen_mb;
    return FAVEST_OK;
}

long long favest_batch_field_elems(favest_batch batch) { return batch ? batch->field_elems : (long long)FAVEST_EINVAL; }
long long favest_batch_coef_elems(favest_batch batch) { return batch ? batch->coef_elems : (long long)FAVEST_EINVAL; }

int favest_batch_status(favest_batch batch, void *stream)
{
    if (!batch) return FAVEST_EINVAL;
    int st = 0;
    for (auto p : batch->groups) {
        int v = favest_status(p, stream);
        if (v != 0 && st == 0) st = v;
    }
    if (batch->d_status) {
        int v = 0;
        if (cudaMemcpy(&v, batch->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return FAVEST_ECUDA;
        if (v != 0) {
            cudaMemset(batch->d_status, 0, sizeof(int));
            if (st == 0) st = v;
        }
    }
    return st;
}

void favest_batch_destroy(favest_batch batch)
{
    if (batch) destroy_batch(batch);
}

}  // extern "C"
