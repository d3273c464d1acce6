// serve.cu -- continuous-batching server for encrypted inference requests.
//
// A model is a program over a request's registers (register 0 holds the
// input and, at the end, the output): a step applies a prepared layer
// (bootstraps included), adds two registers at a level, or multiplies one by
// a constant rescaled onto the model's scale.  A chain of layers is the
// program of one layer step per layer on register 0; a residual network uses
// more registers.  One server takes requests of models on any number of
// contexts (each context with its evaluation keys resident and its own
// stream): LeNet-5 at N = 2^15 and ResNet-20 at N = 2^16 share it.
//
// Admission.  A request's device footprint is its registers, the working
// set one more input adds to each distinct layer of its model (a layer keeps
// one set per input of the largest batch it ran) and the largest
// key-switching workspace one input of a layer's batch needs.  Requests are
// admitted in arrival order while fewer than `max_active` are in flight and
// the footprints of the admitted ones fit the server's memory budget; a
// request that does not fit keeps the later requests of its model waiting,
// while those of other models may pass it; with nothing in flight the oldest
// is admitted whatever its size.  Keys are resident before serving and are
// not part of the budget.
//
// Scheduling.  Each step takes, on every context with requests in flight,
// the stage (model, next step) of its oldest request, and runs that step for
// every admitted request at the same stage -- a layer step as one batch
// (fheon_layer_apply_batch: their rotations share launches) -- on that
// context's stream; the contexts' batches are enqueued one after the other
// and then waited for, so the work of different contexts overlaps on the
// device.  Requests past their model's last step are done and keep their
// result until it is taken.  A request's result is the one the model gives
// its input alone, bit for bit: batching and overlap change launches, never
// arithmetic.  With an admission timeout, a request still waiting that long
// after its submission is dropped at the next admission and its result
// reports FHEON_ERR_TIMEOUT.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <deque>
#include <map>
#include <memory>
#include <set>
#include <vector>

#include "layer.h"

using namespace fheon;

struct fheon_model {
    fheon_ctx *ctx = nullptr;
    std::vector<fheon_step> steps;
    u32 nreg = 1;
    double scale = 0; // target of constant steps
    mutable std::map<u32, size_t> footprint; // by input level
};

namespace {
size_t ct_bytes(const fheon_ctx *ctx, u32 level) { return (size_t)2 * level * ctx->N * 8; }

// key-switching workspace of n rotations at level l hoisted from one input
// (the leader raises the digits, the others keep their own sums), in bytes
size_t ks_bytes(const fheon_ctx *ctx, u32 l, size_t hoisted, size_t plain)
{
    const size_t own = 2 * (size_t)(l + ctx->K) + 2 * (size_t)ctx->K + 2 * (size_t)l;
    size_t limbs = plain * ctx->ks_ws_limbs(l);
    if (hoisted) limbs += ctx->ks_ws_limbs(l) + (hoisted - 1) * own;
    return limbs * ctx->limb_bytes();
}

// what one more input adds to a layer: the working ciphertexts it keeps (one
// set per input of the largest batch it has run) in *work, and the
// key-switching workspace its batch needs per input in *ws
void layer_cost(const fheon_ctx *ctx, const fheon_layer *ly, size_t *work, size_t *ws)
{
    auto series = [&](u32 D, u32 level) {
        u32 k = 1;
        while (k * k < D + 1) k *= 2; // baby steps: 2^ceil(log2(D+1)/2)
        u32 m = 0;
        while ((size_t)k << m <= D) m++;
        return ((size_t)std::min(k, D) + 3 * (size_t)m + 4) * ct_bytes(ctx, level);
    };
    *work = *ws = 0;
    switch (ly->kind) {
    case LAYER_LINEAR: {
        size_t taps = 0;
        for (int32_t r : ly->r) taps += r != 0;
        const size_t groups = std::min<size_t>(ly->s.size(), 32);
        const size_t fold = ly->fold.empty() ? 0 : ly->fold.size() + 1;
        *work = (taps + 2 * groups + fold) * ct_bytes(ctx, ly->level);
        *ws = std::max(ks_bytes(ctx, ly->level, taps, 0), ks_bytes(ctx, ly->level - 1, 0, groups));
        return;
    }
    case LAYER_FC:
        *work = 2 * ly->fw.size() * ct_bytes(ctx, ly->level);
        *ws = ks_bytes(ctx, ly->level - 1, 0, ly->fw.size());
        return;
    case LAYER_CONV:
        *work = ((size_t)ly->k * ly->k + 2) * ct_bytes(ctx, ly->level);
        *ws = ks_bytes(ctx, ly->level, (size_t)ly->k * ly->k - 1, 0);
        return;
    case LAYER_RELU:
        *work = series(ly->degree ? ly->degree : (u32)ly->coeffs.size() - 1, ly->level) + ct_bytes(ctx, ly->level);
        *ws = ks_bytes(ctx, ly->level, 0, 1) + 3 * (size_t)ly->level * ctx->limb_bytes();
        return;
    case LAYER_BOOT: {
        size_t w = 0;
        for (const fheon_layer *l : ly->subs) {
            size_t a, b;
            layer_cost(ctx, l, &a, &b);
            *work += a;
            w = std::max(w, b);
        }
        *work += 10 * ct_bytes(ctx, ctx->L) + 2 * series((u32)ly->coeffs.size() - 1, ctx->L);
        *ws = std::max(w, 2 * ks_bytes(ctx, ctx->L, 0, 1));
        return;
    }
    default: return;
    }
}
} // namespace

namespace {
// a request's buffers: its registers, a step's output and an operand copy;
// `order` remembers the registers' first assignment (steps swap them), so a
// set handed on to a later request starts from the same buffers
struct RegSet {
    std::vector<fheon_ct *> reg;
    fheon_ct *nxt = nullptr, *aux = nullptr;
    std::vector<fheon_ct *> order;
    void restore()
    {
        for (size_t i = 0; i < reg.size(); i++) reg[i] = order[i];
        nxt = order[reg.size()];
    }
    void destroy()
    {
        for (fheon_ct *c : order) fheon_ct_destroy(c);
        fheon_ct_destroy(aux);
        reg.clear();
        order.clear();
        nxt = aux = nullptr;
    }
};

struct Request {
    uint64_t id = 0, seq = 0;
    const fheon_model *model = nullptr;
    size_t footprint = 0;
    u32 next = 0;                 // next step
    std::vector<fheon_ct *> reg;  // registers
    fheon_ct *nxt = nullptr, *aux = nullptr; // a step's output and an operand copy
    std::vector<fheon_ct *> order; // the buffers' first assignment (reg then nxt)
    bool done = false;
    int status = FHEON_OK; // FHEON_ERR_TIMEOUT: dropped before admission
    std::chrono::steady_clock::time_point submitted;
    RegSet take()
    {
        RegSet r{reg, nxt, aux, order};
        reg.clear();
        order.clear();
        nxt = aux = nullptr;
        return r;
    }
    ~Request()
    {
        for (fheon_ct *c : order) fheon_ct_destroy(c);
        fheon_ct_destroy(aux);
    }
};

// one non-layer step of one request: its output into r->nxt
int run_step(fheon_ctx *ctx, const fheon_model *m, const fheon_step &st, Request *r)
{
    int rc;
    if (st.op == FHEON_STEP_ADD) {
        if ((rc = fheon_drop_level(ctx, r->reg[st.src], st.level, r->aux))) return rc;
        if ((rc = fheon_drop_level(ctx, r->reg[st.src2], st.level, r->nxt))) return rc;
        return fheon_add(ctx, r->aux, r->nxt, r->nxt);
    }
    return fheon_mul_const_rescale(ctx, r->reg[st.src], st.c, m->scale, r->nxt);
}
} // namespace

struct fheon_server {
    fheon_ctx *ctx = nullptr; // the context errors are reported on
    u32 max_active = 1;
    size_t budget = 0;        // bytes the admitted requests' footprints may take; 0: no limit
    size_t held = 0;          // footprints of the admitted requests
    std::deque<Request *> waiting;
    std::vector<Request *> active;
    std::map<uint64_t, std::unique_ptr<Request>> all;
    uint64_t next_id = 1, next_seq = 0, steps = 0, mem_waits = 0;
    u32 max_batch = 0;
    std::map<const fheon_model *, u32> model_max_batch;
    double admit_timeout = 0; // seconds a request may wait for admission; 0: no limit
    // graph replay: a layer step of one request runs as the layer's captured
    // graph on that request's buffers, which go back to a per-model pool when
    // the result is taken, so the next request of the model replays them
    bool graphs = false;
    std::map<const fheon_model *, std::vector<RegSet>> pool;
    uint64_t replays = 0;
    ~fheon_server()
    {
        for (auto &kv : pool)
            for (RegSet &r : kv.second) r.destroy();
    }
};

namespace {
// drop the waiting requests past the admission timeout (counted in *expired),
// then admit what fits
int admit(fheon_server *s, u32 *expired)
{
    if (s->admit_timeout > 0) {
        const auto now = std::chrono::steady_clock::now();
        for (auto it = s->waiting.begin(); it != s->waiting.end();) {
            Request *r = *it;
            if (std::chrono::duration<double>(now - r->submitted).count() > s->admit_timeout) {
                r->done = true;
                r->status = FHEON_ERR_TIMEOUT;
                ++*expired;
                it = s->waiting.erase(it);
            } else {
                ++it;
            }
        }
    }
    std::set<const fheon_model *> blocked; // models whose oldest waiting request did not fit
    for (auto it = s->waiting.begin(); it != s->waiting.end() && s->active.size() < s->max_active;) {
        Request *r = *it;
        if (blocked.count(r->model)) {
            ++it;
            continue;
        }
        if (s->budget && s->held + r->footprint > s->budget && !s->active.empty()) {
            blocked.insert(r->model);
            s->mem_waits++;
            ++it;
            continue;
        }
        it = s->waiting.erase(it);
        r->seq = s->next_seq++;
        s->held += r->footprint;
        s->active.push_back(r);
    }
    return FHEON_OK;
}
} // namespace

extern "C" {

int fheon_model_create_program(fheon_ctx *ctx, const fheon_step *steps, uint32_t n, uint32_t nreg, double scale,
                               fheon_model **out)
{
    if (!ctx || !out || !n || !steps || !nreg || nreg > 64) return FHEON_ERR_ARG;
    for (u32 i = 0; i < n; i++) {
        const fheon_step &st = steps[i];
        const bool regs_ok = st.src < nreg && st.dst < nreg && (st.op != FHEON_STEP_ADD || st.src2 < nreg);
        if (!regs_ok) return fail(ctx, FHEON_ERR_ARG, "model step %u: register out of range", i);
        if (st.op == FHEON_STEP_LAYER && !st.layer) return fail(ctx, FHEON_ERR_ARG, "model step %u: no layer", i);
        if (st.op == FHEON_STEP_ADD && st.level < 1) return fail(ctx, FHEON_ERR_ARG, "model step %u: level 0", i);
        if (st.op == FHEON_STEP_SCALE && !(scale > 0)) return fail(ctx, FHEON_ERR_ARG, "model step %u: no scale", i);
        if (st.op > FHEON_STEP_SCALE) return fail(ctx, FHEON_ERR_ARG, "model step %u: unknown op %u", i, st.op);
    }
    fheon_model *m = new fheon_model();
    m->ctx = ctx;
    m->steps.assign(steps, steps + n);
    m->nreg = nreg;
    m->scale = scale;
    *out = m;
    return FHEON_OK;
}

int fheon_model_create(fheon_ctx *ctx, const fheon_layer *const *layers, uint32_t n, fheon_model **out)
{
    if (!ctx || !out || !n || !layers) return FHEON_ERR_ARG;
    std::vector<fheon_step> st(n);
    for (u32 i = 0; i < n; i++) {
        if (!layers[i]) return FHEON_ERR_ARG;
        st[i] = fheon_step{FHEON_STEP_LAYER, 0, 0, 0, 0, layers[i], 0.0};
    }
    return fheon_model_create_program(ctx, st.data(), n, 1, 0.0, out);
}

int fheon_model_run(fheon_ctx *ctx, const fheon_model *m, const fheon_ct *in, fheon_ct *out)
{
    if (!ctx || !m || !in || !out || m->ctx != ctx) return FHEON_ERR_ARG;
    Request r;
    r.model = m;
    r.reg.assign(m->nreg, nullptr);
    int rc;
    for (fheon_ct *&c : r.reg) {
        if ((rc = fheon_ct_create(ctx, in->level, in->scale, &c))) return rc;
        r.order.push_back(c);
    }
    if ((rc = fheon_ct_create(ctx, in->level, in->scale, &r.nxt))) return rc;
    r.order.push_back(r.nxt);
    if ((rc = fheon_ct_create(ctx, in->level, in->scale, &r.aux))) return rc;
    if ((rc = fheon_drop_level(ctx, in, in->level, r.reg[0]))) return rc;
    for (const fheon_step &st : m->steps) {
        if (st.op == FHEON_STEP_LAYER) {
            if ((rc = fheon_layer_apply(ctx, st.layer, r.reg[st.src], r.nxt))) return rc;
        } else if ((rc = run_step(ctx, m, st, &r))) {
            return rc;
        }
        std::swap(r.reg[st.dst], r.nxt);
    }
    rc = fheon_drop_level(ctx, r.reg[0], r.reg[0]->level, out);
    if (!rc) rc = fheon_sync(ctx); // the request's buffers go with it
    return rc;
}

int fheon_model_destroy(fheon_model *m)
{
    delete m;
    return FHEON_OK;
}

int fheon_model_footprint(const fheon_model *m, uint32_t level, size_t *bytes)
{
    if (!m || !bytes || level < 1 || level > m->ctx->L) return FHEON_ERR_ARG;
    auto it = m->footprint.find(level);
    if (it == m->footprint.end()) {
        // every distinct layer keeps its own working set; the workspace is shared
        std::set<const fheon_layer *> seen;
        size_t work = 0, ws = 0;
        for (const fheon_step &st : m->steps)
            if (st.op == FHEON_STEP_LAYER && seen.insert(st.layer).second) {
                size_t a, b;
                layer_cost(m->ctx, st.layer, &a, &b);
                work += a;
                ws = std::max(ws, b);
            }
        it = m->footprint.emplace(level, (size_t)(m->nreg + 2) * ct_bytes(m->ctx, level) + work + ws).first;
    }
    *bytes = it->second;
    return FHEON_OK;
}

int fheon_server_create(fheon_ctx *ctx, uint32_t max_active, size_t mem_budget, fheon_server **out)
{
    if (!ctx || !out || !max_active) return FHEON_ERR_ARG;
    fheon_server *s = new fheon_server();
    s->ctx = ctx;
    s->max_active = max_active;
    s->budget = mem_budget;
    *out = s;
    return FHEON_OK;
}

int fheon_server_destroy(fheon_server *s)
{
    if (s) {
        std::set<fheon_ctx *> ctxs{s->ctx};
        for (auto &kv : s->all) ctxs.insert(kv.second->model->ctx);
        for (fheon_ctx *c : ctxs)
            if (c) cudaStreamSynchronize(c->stream);
    }
    delete s;
    return FHEON_OK;
}

int fheon_server_submit(fheon_server *s, const fheon_model *m, const fheon_ct *in, uint64_t *id)
{
    if (!s || !m || !in || !id) return FHEON_ERR_ARG;
    fheon_ctx *ctx = m->ctx;
    std::unique_ptr<Request> r(new Request());
    int rc;
    if ((rc = fheon_model_footprint(m, in->level, &r->footprint))) return rc;
    auto pit = s->pool.find(m);
    if (s->graphs && pit != s->pool.end() && !pit->second.empty()) {
        RegSet set = pit->second.back();
        pit->second.pop_back();
        r->reg = set.reg;
        r->nxt = set.nxt;
        r->aux = set.aux;
        r->order = set.order;
    } else {
        r->reg.assign(m->nreg, nullptr);
        for (fheon_ct *&c : r->reg) {
            if ((rc = fheon_ct_create(ctx, in->level, in->scale, &c))) return rc;
            r->order.push_back(c);
        }
        if ((rc = fheon_ct_create(ctx, in->level, in->scale, &r->nxt))) return rc;
        r->order.push_back(r->nxt);
        if ((rc = fheon_ct_create(ctx, in->level, in->scale, &r->aux))) return rc;
    }
    if ((rc = fheon_drop_level(ctx, in, in->level, r->reg[0]))) return rc; // the request's own copy
    r->id = s->next_id++;
    r->model = m;
    r->submitted = std::chrono::steady_clock::now();
    *id = r->id;
    s->waiting.push_back(r.get());
    s->all.emplace(r->id, std::move(r));
    return FHEON_OK;
}

int fheon_server_step(fheon_server *s, uint32_t *n_done)
{
    if (!s) return FHEON_ERR_ARG;
    Range range("server_step");
    if (n_done) *n_done = 0;
    u32 expired = 0;
    int rc = admit(s, &expired);
    if (n_done) *n_done = expired;
    if (rc) return rc;
    if (s->active.empty()) return FHEON_OK;
    // per context: the oldest request's stage, and every request at it
    std::map<fheon_ctx *, const Request *> oldest;
    for (const Request *r : s->active) {
        auto it = oldest.find(r->model->ctx);
        if (it == oldest.end() || r->seq < it->second->seq) oldest[r->model->ctx] = r;
    }
    std::vector<std::vector<Request *>> batches;
    for (auto &kv : oldest) {
        const fheon_model *m = kv.second->model;
        const u32 stage = kv.second->next;
        std::vector<Request *> batch;
        for (Request *r : s->active)
            if (r->model == m && r->next == stage) batch.push_back(r);
        fheon_ctx *ctx = kv.first;
        const fheon_step &st = m->steps[stage];
        if (st.op == FHEON_STEP_LAYER && s->graphs && batch.size() == 1) {
            rc = fheon_layer_apply_graph(ctx, st.layer, batch[0]->reg[st.src], batch[0]->nxt);
            s->replays++;
        } else if (st.op == FHEON_STEP_LAYER) {
            std::vector<const fheon_ct *> ins;
            std::vector<fheon_ct *> outs;
            for (Request *r : batch) {
                ins.push_back(r->reg[st.src]);
                outs.push_back(r->nxt);
            }
            rc = fheon_layer_apply_batch(ctx, st.layer, ins.data(), (u32)batch.size(), outs.data());
        } else {
            for (Request *r : batch)
                if ((rc = run_step(ctx, m, st, r))) break;
        }
        if (rc) {
            if (ctx != s->ctx) s->ctx->last_error = ctx->last_error; // reported on the server's context
            return rc;
        }
        s->max_batch = std::max<u32>(s->max_batch, (u32)batch.size());
        u32 &mb = s->model_max_batch[m];
        mb = std::max<u32>(mb, (u32)batch.size());
        batches.push_back(std::move(batch));
    }
    s->steps++;
    // wait for every context's batch (they ran concurrently on their streams)
    for (auto &kv : oldest)
        if ((rc = fheon_sync(kv.first))) return rc;
    u32 done = 0;
    for (auto &batch : batches)
        for (Request *r : batch) {
            const fheon_step &st = r->model->steps[r->next];
            std::swap(r->reg[st.dst], r->nxt);
            r->next++;
            if (r->next == r->model->steps.size()) {
                r->done = true;
                s->held -= r->footprint;
                done++;
            }
        }
    s->active.erase(std::remove_if(s->active.begin(), s->active.end(), [](const Request *r) { return r->done; }),
                    s->active.end());
    if (n_done) *n_done = done + expired;
    return FHEON_OK;
}

int fheon_server_result(fheon_server *s, uint64_t id, fheon_ct *out)
{
    if (!s || !out) return FHEON_ERR_ARG;
    auto it = s->all.find(id);
    if (it == s->all.end()) return fail(s->ctx, FHEON_ERR_ARG, "no request %llu", (unsigned long long)id);
    if (it->second->status != FHEON_OK) {
        const int st = it->second->status;
        s->all.erase(it);
        return fail(s->ctx, st, "request %llu waited longer than the admission timeout", (unsigned long long)id);
    }
    if (!it->second->done) return FHEON_PENDING;
    const fheon_ct *r = it->second->reg[0];
    fheon_ctx *ctx = it->second->model->ctx;
    int rc = fheon_drop_level(ctx, r, r->level, out);
    if (rc) return rc;
    if ((rc = fheon_sync(ctx))) return rc;
    if (s->graphs) {
        // the buffers serve the model's next request (its graphs replay on them)
        RegSet set = it->second->take();
        set.restore();
        s->pool[it->second->model].push_back(set);
    }
    s->all.erase(it);
    return FHEON_OK;
}

int fheon_server_set_graphs(fheon_server *s, int on)
{
    if (!s) return FHEON_ERR_ARG;
    std::set<fheon_ctx *> ctxs{s->ctx};
    for (auto &kv : s->all) ctxs.insert(kv.second->model->ctx);
    for (fheon_ctx *c : ctxs)
        if (on && c && !c->stream)
            return fail(s->ctx, FHEON_ERR_ARG, "graph replay needs created streams, not the legacy default stream");
    if (!on)
        for (auto &kv : s->pool)
            for (RegSet &r : kv.second) r.destroy();
    if (!on) s->pool.clear();
    s->graphs = on != 0;
    return FHEON_OK;
}

int fheon_server_graph_replays(const fheon_server *s, uint64_t *replays)
{
    if (!s || !replays) return FHEON_ERR_ARG;
    *replays = s->replays;
    return FHEON_OK;
}

int fheon_server_set_admit_timeout(fheon_server *s, double seconds)
{
    if (!s || !(seconds >= 0) || std::isinf(seconds)) return FHEON_ERR_ARG;
    s->admit_timeout = seconds;
    return FHEON_OK;
}

int fheon_server_stats(const fheon_server *s, uint64_t *steps, uint32_t *max_batch, uint32_t *active,
                       uint32_t *waiting)
{
    if (!s) return FHEON_ERR_ARG;
    if (steps) *steps = s->steps;
    if (max_batch) *max_batch = s->max_batch;
    if (active) *active = (uint32_t)s->active.size();
    if (waiting) *waiting = (uint32_t)s->waiting.size();
    return FHEON_OK;
}

int fheon_server_model_stats(const fheon_server *s, const fheon_model *m, uint32_t *max_batch, uint64_t *mem_waits,
                             size_t *held)
{
    if (!s || !m) return FHEON_ERR_ARG;
    auto it = s->model_max_batch.find(m);
    if (max_batch) *max_batch = it == s->model_max_batch.end() ? 0 : it->second;
    if (mem_waits) *mem_waits = s->mem_waits;
    if (held) *held = s->held;
    return FHEON_OK;
}

} // extern "C"
