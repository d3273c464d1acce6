// serve.cu -- continuous-batching server for encrypted inference requests.
//
// Requests of one or more models (ordered lists of prepared layers on one
// context, evaluation keys resident) arrive over time.  A request is admitted
// while fewer than `max_active` are in flight and the device has at least
// `min_free` bytes free; the rest wait in arrival order.  Each step takes the
// oldest admitted request's stage (model, next layer), applies that layer to
// every admitted request at the same stage as one batch
// (fheon_layer_apply_batch: their rotations share launches), and advances
// them; requests past their model's last layer are done and keep their result
// until it is taken.  A request's result is the one the model gives its input
// alone, bit for bit: batching changes launches, never arithmetic.
#include <algorithm>
#include <deque>
#include <map>
#include <memory>
#include <vector>

#include "layer.h"

using namespace fheon;

struct fheon_model {
    fheon_ctx *ctx = nullptr;
    std::vector<const fheon_layer *> layers;
};

namespace {
struct Request {
    uint64_t id = 0, seq = 0;
    const fheon_model *model = nullptr;
    u32 next = 0; // next layer
    fheon_ct *cur = nullptr, *nxt = nullptr;
    bool done = false;
    ~Request()
    {
        fheon_ct_destroy(cur);
        fheon_ct_destroy(nxt);
    }
};
} // namespace

struct fheon_server {
    fheon_ctx *ctx = nullptr;
    u32 max_active = 1;
    size_t min_free = 0;
    std::deque<Request *> waiting;
    std::vector<Request *> active;
    std::map<uint64_t, std::unique_ptr<Request>> all;
    uint64_t next_id = 1, next_seq = 0, steps = 0;
    u32 max_batch = 0;
};

namespace {
int admit(fheon_server *s)
{
    while (!s->waiting.empty() && s->active.size() < s->max_active) {
        if (s->min_free) {
            size_t free_b = 0, total_b = 0;
            FHEON_CUDA(s->ctx, cudaMemGetInfo(&free_b, &total_b));
            if (free_b < s->min_free && !s->active.empty()) break; // the oldest always gets in
        }
        Request *r = s->waiting.front();
        s->waiting.pop_front();
        r->seq = s->next_seq++;
        s->active.push_back(r);
    }
    return FHEON_OK;
}
} // namespace

extern "C" {

int fheon_model_create(fheon_ctx *ctx, const fheon_layer *const *layers, uint32_t n, fheon_model **out)
{
    if (!ctx || !out || !n || !layers) return FHEON_ERR_ARG;
    for (u32 i = 0; i < n; i++)
        if (!layers[i]) return FHEON_ERR_ARG;
    fheon_model *m = new fheon_model();
    m->ctx = ctx;
    m->layers.assign(layers, layers + n);
    *out = m;
    return FHEON_OK;
}

int fheon_model_destroy(fheon_model *m)
{
    delete m;
    return FHEON_OK;
}

int fheon_server_create(fheon_ctx *ctx, uint32_t max_active, size_t min_free, fheon_server **out)
{
    if (!ctx || !out || !max_active) return FHEON_ERR_ARG;
    fheon_server *s = new fheon_server();
    s->ctx = ctx;
    s->max_active = max_active;
    s->min_free = min_free;
    *out = s;
    return FHEON_OK;
}

int fheon_server_destroy(fheon_server *s)
{
    if (s && s->ctx) cudaStreamSynchronize(s->ctx->stream);
    delete s;
    return FHEON_OK;
}

int fheon_server_submit(fheon_server *s, const fheon_model *m, const fheon_ct *in, uint64_t *id)
{
    if (!s || !m || !in || !id || m->ctx != s->ctx) return FHEON_ERR_ARG;
    std::unique_ptr<Request> r(new Request());
    int rc;
    if ((rc = fheon_ct_create(s->ctx, in->level, in->scale, &r->cur))) return rc;
    if ((rc = fheon_ct_create(s->ctx, in->level, in->scale, &r->nxt))) return rc;
    if ((rc = fheon_drop_level(s->ctx, in, in->level, r->cur))) return rc; // the request's own copy
    r->id = s->next_id++;
    r->model = m;
    *id = r->id;
    s->waiting.push_back(r.get());
    s->all.emplace(r->id, std::move(r));
    return FHEON_OK;
}

int fheon_server_step(fheon_server *s, uint32_t *n_done)
{
    if (!s) return FHEON_ERR_ARG;
    if (n_done) *n_done = 0;
    int rc = admit(s);
    if (rc) return rc;
    if (s->active.empty()) return FHEON_OK;
    const Request *oldest = *std::min_element(s->active.begin(), s->active.end(),
                                              [](const Request *a, const Request *b) { return a->seq < b->seq; });
    const fheon_model *m = oldest->model;
    const u32 stage = oldest->next;
    std::vector<Request *> batch;
    for (Request *r : s->active)
        if (r->model == m && r->next == stage) batch.push_back(r);
    std::vector<const fheon_ct *> ins;
    std::vector<fheon_ct *> outs;
    for (Request *r : batch) {
        ins.push_back(r->cur);
        outs.push_back(r->nxt);
    }
    if ((rc = fheon_layer_apply_batch(s->ctx, m->layers[stage], ins.data(), (u32)batch.size(), outs.data()))) return rc;
    s->steps++;
    s->max_batch = std::max<u32>(s->max_batch, (u32)batch.size());
    u32 done = 0;
    for (Request *r : batch) {
        std::swap(r->cur, r->nxt);
        r->next++;
        if (r->next == m->layers.size()) {
            r->done = true;
            done++;
        }
    }
    s->active.erase(std::remove_if(s->active.begin(), s->active.end(), [](const Request *r) { return r->done; }),
                    s->active.end());
    if ((rc = fheon_sync(s->ctx))) return rc;
    if (n_done) *n_done = done;
    return FHEON_OK;
}

int fheon_server_result(fheon_server *s, uint64_t id, fheon_ct *out)
{
    if (!s || !out) return FHEON_ERR_ARG;
    auto it = s->all.find(id);
    if (it == s->all.end()) return fail(s->ctx, FHEON_ERR_ARG, "no request %llu", (unsigned long long)id);
    if (!it->second->done) return FHEON_PENDING;
    const fheon_ct *r = it->second->cur;
    int rc = fheon_drop_level(s->ctx, r, r->level, out);
    if (rc) return rc;
    if ((rc = fheon_sync(s->ctx))) return rc;
    s->all.erase(it);
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

} // extern "C"
