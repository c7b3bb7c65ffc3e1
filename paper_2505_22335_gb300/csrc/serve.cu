// Request queue with continuous batching (include/ups.h, "serving").
//
// Each slot is a worker thread with its own ups_ctx, CUDA stream and batch
// buffers.  A worker takes the requests waiting in the queue (FIFO) as long as
// they fit in max_batch_views and in the memory budget, concatenates their
// views (tracking: the pyramid levels of one pose; mapping: its keyframes) and
// runs one decode -> forward -> per-request loss -> backward -> per-request
// decode backward on its stream.  Several slots keep several batches on the
// GPU at once; a stream host-callback stamps completion and releases the
// batch's memory reservation, which admits the next batch.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "common.cuh"

namespace ups {
ups_status loss_views(ups_ctx *c, const ups_images *img, const ups_targets *tgt,
                      const ups_loss_cfg *lcfg, int v0, int v1, float *loss_dev, ups_images *dL,
                      cudaStream_t st);
ups_status render_forward_sets(ups_ctx *c, const ups_gaussians *g, const ups_camera *cams, int n_views,
                               const int *set_of_view, ups_images *out, ups_stream stream);
}

using namespace ups;

namespace {

__global__ void k_sum_pose(const float *__restrict__ in, int levels, float *__restrict__ out) {
    const int i = threadIdx.x;
    if (i < 6) {
        float s = 0.f;
        for (int l = 0; l < levels; ++l) s += in[6 * l + i];
        out[i] = s;
    }
}

struct Buf {
    void *p = nullptr;
    size_t n = 0;
    cudaError_t reserve(size_t b) {
        if (b <= n) return cudaSuccess;
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
        size_t want = std::max<size_t>(b + b / 8, 256);
        cudaError_t e = cudaMalloc(&p, want);
        if (e == cudaSuccess) n = want;
        return e;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
    template <class T> T *as() const { return static_cast<T *>(p); }
};

struct Req {
    uint64_t ticket = 0;
    ups_request r{};
    std::vector<ups_camera> cams;  // effective views (tracking: one per level)
    int nv = 0;
    size_t pixels = 0, bytes = 0;
    int status = UPS_PENDING;
    bool started = false;
    double t_submit = 0, t_start = 0, t_end = 0;
    int batch_id = -1, batch_reqs = 0, batch_views = 0;
    int anc_n = 0;  // anchors of the scene at submission (the size of d_anchors)
};

struct Slot {
    ups_ctx *ctx = nullptr;
    cudaStream_t st = nullptr;
    Buf g[5], dg[5];          // decoded sets and their gradients: mean|o, scale, quat, colour, feature
    Buf im[5], dl[3], pose;   // images (colour, depth, feature, T, n_contrib), image grads, pose grads
};

}  // namespace

struct ups_server {
    ups_config cfg{};
    ups_server_config scfg{};
    int device = 0;
    ups_anchors anc{};
    ups_mlp mlp{};
    std::vector<Slot> slots;
    std::vector<std::thread> workers;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Req *> queue;
    std::unordered_map<uint64_t, Req *> reqs;
    bool stopping = false;
    bool paused = false;  // ups_server_set_scene: no new batch starts
    uint64_t next_ticket = 1;
    int next_batch = 0;
    size_t reserved = 0, budget = 0;
    int in_flight = 0;
    std::chrono::steady_clock::time_point t0;
    std::string err;
    double now_ms() const {
        return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
};

namespace {

struct BatchDone {
    ups_server *srv;
    std::vector<Req *> reqs;
    size_t bytes;
};

void CUDART_CB on_batch_done(void *p) {
    BatchDone *bd = static_cast<BatchDone *>(p);
    ups_server *s = bd->srv;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        const double t = s->now_ms();
        for (Req *r : bd->reqs) {
            r->t_end = t;
            if (r->status == UPS_PENDING) r->status = UPS_OK;
        }
        s->reserved -= bd->bytes;
        s->in_flight--;
    }
    s->cv.notify_all();
    delete bd;
}

void finish_now(ups_server *s, std::vector<Req *> &batch, size_t bytes, int status) {
    {
        std::lock_guard<std::mutex> lk(s->mu);
        const double t = s->now_ms();
        for (Req *r : batch) {
            r->t_end = t;
            r->status = status;
        }
        s->reserved -= bytes;
        s->in_flight--;
    }
    s->cv.notify_all();
}

size_t footprint(const ups_config &c, size_t n_gauss, int nv, size_t pixels) {
    const size_t per_gv = 2 * (64 + 4 * (size_t)c.n_feat) + 120 + 10 * 16;
    return (size_t)nv * n_gauss * per_gv + pixels * (8 * (5 + (size_t)c.n_feat) + 8);
}

// one batched step; returns UPS_OK when queued on the stream.  The decode
// (Eq. 8-9) depends on a view only through its camera centre and time, so the
// pyramid levels of a tracking request share one decoded set: the batch
// decodes one set per tracking request and one per mapping keyframe, and the
// forward maps each rendered view to its set.
ups_status run_batch(ups_server *s, Slot &sl, std::vector<Req *> &batch, std::string &msg) {
    std::vector<ups_camera> cams, dcams;  // rendered views; decoded sets
    std::vector<int> v0, s0, set_of_view;
    size_t P = 0;
    for (Req *r : batch) {
        v0.push_back((int)cams.size());
        s0.push_back((int)dcams.size());
        cams.insert(cams.end(), r->cams.begin(), r->cams.end());
        if (r->r.kind == UPS_REQ_TRACK) {
            dcams.push_back(r->cams[0]);
            for (int l = 0; l < r->nv; ++l) set_of_view.push_back(s0.back());
        } else {
            for (int k = 0; k < r->nv; ++k) {
                dcams.push_back(r->cams[k]);
                set_of_view.push_back(s0.back() + k);
            }
        }
        P += r->pixels;
    }
    const int V = (int)cams.size(), S = (int)dcams.size();
    const int NF = s->cfg.n_feat;
    const size_t N = (size_t)s->anc.n * s->cfg.k;
    const size_t GV = (size_t)S * N;
    cudaError_t e = cudaSuccess;
    const size_t rec[5] = {16, 16, 16, 16, 4 * (size_t)NF};
    for (int i = 0; i < 5 && e == cudaSuccess; ++i) {
        e = sl.g[i].reserve(std::max<size_t>(GV * rec[i], 16));
        if (e == cudaSuccess) e = sl.dg[i].reserve(std::max<size_t>(GV * rec[i], 16));
    }
    const size_t imsz[5] = {12 * P, 4 * P, 4 * (size_t)NF * P, 4 * P, 4 * P};
    for (int i = 0; i < 5 && e == cudaSuccess; ++i) e = sl.im[i].reserve(std::max<size_t>(imsz[i], 16));
    for (int i = 0; i < 3 && e == cudaSuccess; ++i) e = sl.dl[i].reserve(std::max<size_t>(imsz[i], 16));
    if (e == cudaSuccess) e = sl.pose.reserve((size_t)V * 6 * 4);
    if (e != cudaSuccess) {
        msg = std::string("batch buffers: ") + cudaGetErrorString(e);
        return UPS_ERR_OOM;
    }
    ups_gaussians G{(int)N, 1, sl.g[0].as<float>(), sl.g[1].as<float>(), sl.g[2].as<float>(),
                    sl.g[3].as<float>(), NF ? sl.g[4].as<float>() : nullptr};
    ups_gaussians dG{(int)N, 1, sl.dg[0].as<float>(), sl.dg[1].as<float>(), sl.dg[2].as<float>(),
                     sl.dg[3].as<float>(), NF ? sl.dg[4].as<float>() : nullptr};
    ups_images img{sl.im[0].as<float>(), sl.im[1].as<float>(), NF ? sl.im[2].as<float>() : nullptr,
                   sl.im[3].as<float>(), sl.im[4].as<uint32_t>()};
    ups_images dl{sl.dl[0].as<float>(), sl.dl[1].as<float>(), NF ? sl.dl[2].as<float>() : nullptr,
                  nullptr, nullptr};
    float *pose = sl.pose.as<float>();
    ups_status st = ups_decode_anchors(sl.ctx, &s->anc, &s->mlp, dcams.data(), S, &G, sl.st);
    if (st == UPS_OK) st = render_forward_sets(sl.ctx, &G, cams.data(), V, set_of_view.data(), &img, sl.st);
    for (size_t i = 0; i < batch.size() && st == UPS_OK; ++i)
        st = loss_views(sl.ctx, &img, &batch[i]->r.targets, &s->scfg.loss, v0[i], v0[i] + batch[i]->nv,
                        batch[i]->r.loss, &dl, sl.st);
    if (st == UPS_OK) {
        ups_image_grads g{dl.color, dl.depth, dl.feat, nullptr};
        st = ups_render_backward(sl.ctx, &g, UPS_GRAD_POSE | UPS_GRAD_GAUSS, 0.f, &dG, pose, sl.st);
    }
    for (size_t i = 0; i < batch.size() && st == UPS_OK; ++i) {
        Req *r = batch[i];
        const size_t off = (size_t)s0[i] * N;
        const int n_sets = r->r.kind == UPS_REQ_TRACK ? 1 : r->nv;
        ups_gaussians dGr{(int)N, 1, dG.mean_opacity + 4 * off, dG.scale + 4 * off, dG.quat + 4 * off,
                          dG.color + 4 * off, NF ? dG.feat + (size_t)NF * off : nullptr};
        unsigned mask = UPS_GRAD_POSE;
        if (r->r.kind == UPS_REQ_MAP && r->r.d_mlp.w1) mask |= UPS_GRAD_MLP;
        if (r->r.kind == UPS_REQ_MAP && r->r.d_anchors.pos) mask |= UPS_GRAD_ANCHOR;
        ups_anchors da = r->r.d_anchors;
        da.n = s->anc.n;
        // the camera-centre part of the pose gradient goes to the request's
        // first view (a tracking request's levels are summed below)
        st = ups_decode_backward(sl.ctx, &s->anc, &s->mlp, dcams.data() + s0[i], n_sets, &dGr, mask,
                                 &r->r.d_mlp, &da, pose + 6 * v0[i], sl.st);
        if (st != UPS_OK) break;
        if (r->r.kind == UPS_REQ_TRACK) {
            k_sum_pose<<<1, 32, 0, sl.st>>>(pose + 6 * v0[i], r->nv, r->r.d_pose);
            e = cudaGetLastError();
        } else {
            e = cudaMemcpyAsync(r->r.d_pose, pose + 6 * v0[i], sizeof(float) * 6 * r->nv,
                                cudaMemcpyDeviceToDevice, sl.st);
        }
        if (e != cudaSuccess) {
            msg = cudaGetErrorString(e);
            return UPS_ERR_CUDA;
        }
    }
    if (st != UPS_OK) msg = ups_last_error(sl.ctx);
    return st;
}

void worker(ups_server *s, int si) {
    cudaSetDevice(s->device);
    Slot &sl = s->slots[si];
    for (;;) {
        std::vector<Req *> batch;
        size_t bytes = 0;
        int views = 0, id = 0;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv.wait(lk, [&] { return s->stopping || (!s->paused && !s->queue.empty()); });
            if (s->queue.empty()) {
                if (s->stopping) return;
                continue;
            }
            if (s->paused && !s->stopping) continue;
            while (!s->queue.empty()) {
                Req *r = s->queue.front();
                if (r->r.kind == UPS_REQ_MAP && r->r.d_anchors.pos && r->anc_n != s->anc.n) {
                    // its anchor-gradient buffers were sized for the scene before the last
                    // ups_server_set_scene: fail it rather than write past them
                    s->queue.pop_front();
                    r->started = true;
                    r->status = UPS_ERR_STATE;
                    r->t_start = r->t_end = s->now_ms();
                    s->err = "mapping request with anchor gradients submitted for a scene of " +
                             std::to_string(r->anc_n) + " anchors, scene now has " + std::to_string(s->anc.n);
                    continue;
                }
                if (!batch.empty() && (!s->scfg.batching || views + r->nv > s->scfg.max_batch_views)) break;
                // admission by memory footprint; an oversized request still runs
                // alone once nothing else is in flight
                if (s->reserved + bytes + r->bytes > s->budget && (!batch.empty() || s->in_flight > 0)) break;
                s->queue.pop_front();
                r->started = true;
                batch.push_back(r);
                views += r->nv;
                bytes += r->bytes;
                if (!s->scfg.batching) break;
            }
            if (batch.empty()) {
                s->cv.wait(lk);
                continue;
            }
            s->reserved += bytes;
            s->in_flight++;
            id = s->next_batch++;
            const double t = s->now_ms();
            for (Req *r : batch) {
                r->t_start = t;
                r->batch_id = id;
                r->batch_reqs = (int)batch.size();
                r->batch_views = views;
            }
        }
        std::string msg;
        ups_status st = run_batch(s, sl, batch, msg);
        if (st == UPS_OK) {
            BatchDone *bd = new BatchDone{s, batch, bytes};
            if (cudaLaunchHostFunc(sl.st, on_batch_done, bd) != cudaSuccess) {
                delete bd;
                cudaStreamSynchronize(sl.st);
                finish_now(s, batch, bytes, UPS_ERR_CUDA);
            }
        } else {
            cudaStreamSynchronize(sl.st);
            {
                std::lock_guard<std::mutex> lk(s->mu);
                s->err = msg;
            }
            finish_now(s, batch, bytes, st);
        }
    }
}

}  // namespace

extern "C" {

ups_status ups_server_create(const ups_config *cfg, const ups_server_config *scfg, int device,
                             const ups_anchors *scene, const ups_mlp *mlp, ups_server **out) {
    if (!cfg || !scfg || !scene || !mlp || !out) return UPS_ERR_ARG;
    *out = nullptr;
    if (scfg->slots < 1 || scfg->slots > 16 || scfg->max_batch_views < 1 ||
        scfg->max_batch_views > UPS_MAX_VIEWS || scene->n < 1 || !scene->pos || !scene->feat ||
        !scene->offsets || !scene->scaling || !mlp->w1 || !mlp->b1 || !mlp->w2 || !mlp->b2)
        return UPS_ERR_ARG;
    ups_server *s = new ups_server();
    s->cfg = *cfg;
    s->scfg = *scfg;
    s->device = device;
    s->anc = *scene;
    s->mlp = *mlp;
    s->budget = (size_t)(std::max(scfg->memory_budget_gb, 0.0) * 1e9);
    s->t0 = std::chrono::steady_clock::now();
    s->slots.resize(scfg->slots);
    ups_status st = UPS_OK;
    if (cudaSetDevice(device) != cudaSuccess) st = UPS_ERR_CUDA;
    for (int i = 0; i < scfg->slots && st == UPS_OK; ++i) {
        st = ups_create(cfg, device, &s->slots[i].ctx);
        if (st == UPS_OK && cudaStreamCreateWithFlags(&s->slots[i].st, cudaStreamNonBlocking) != cudaSuccess)
            st = UPS_ERR_CUDA;
    }
    if (st != UPS_OK) {
        for (Slot &sl : s->slots) {
            if (sl.ctx) ups_destroy(sl.ctx);
            if (sl.st) cudaStreamDestroy(sl.st);
        }
        delete s;
        return st;
    }
    for (int i = 0; i < scfg->slots; ++i) s->workers.emplace_back(worker, s, i);
    *out = s;
    return UPS_OK;
}

ups_status ups_server_destroy(ups_server *s) {
    if (!s) return UPS_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stopping = true;
    }
    s->cv.notify_all();
    for (std::thread &t : s->workers) t.join();
    cudaSetDevice(s->device);
    for (Slot &sl : s->slots) cudaStreamSynchronize(sl.st);
    {
        // host callbacks of the last batches
        std::unique_lock<std::mutex> lk(s->mu);
        s->cv.wait_for(lk, std::chrono::seconds(30), [&] { return s->in_flight == 0; });
    }
    for (Slot &sl : s->slots) {
        for (Buf &b : sl.g) b.release();
        for (Buf &b : sl.dg) b.release();
        for (Buf &b : sl.im) b.release();
        for (Buf &b : sl.dl) b.release();
        sl.pose.release();
        ups_destroy(sl.ctx);
        cudaStreamDestroy(sl.st);
    }
    for (auto &kv : s->reqs) delete kv.second;
    delete s;
    return UPS_OK;
}

ups_status ups_submit(ups_server *s, const ups_request *req, uint64_t *ticket) {
    if (!s || !req || !ticket) return UPS_ERR_ARG;
    if ((req->kind != UPS_REQ_TRACK && req->kind != UPS_REQ_MAP) || !req->cams || !req->loss ||
        !req->d_pose || !req->targets.color || !req->targets.depth ||
        (s->cfg.n_feat > 0 && !req->targets.feat))
        return UPS_ERR_ARG;
    Req *r = new Req();
    r->r = *req;
    if (req->kind == UPS_REQ_TRACK) {
        if (req->levels < 1 || req->levels > 4) {
            delete r;
            return UPS_ERR_ARG;
        }
        for (int l = 0; l < req->levels; ++l) {
            ups_camera c = req->cams[0];
            const float f = 1.f / (float)(1 << l);
            c.fx *= f;
            c.fy *= f;
            c.cx *= f;
            c.cy *= f;
            c.width = std::max(1, req->cams[0].width >> l);
            c.height = std::max(1, req->cams[0].height >> l);
            r->cams.push_back(c);
        }
    } else {
        if (req->n_views < 1 || req->n_views > s->scfg.max_batch_views) {
            delete r;
            return UPS_ERR_ARG;
        }
        r->cams.assign(req->cams, req->cams + req->n_views);
    }
    r->nv = (int)r->cams.size();
    if (r->nv > s->scfg.max_batch_views) {
        delete r;
        return UPS_ERR_ARG;
    }
    for (const ups_camera &c : r->cams) r->pixels += (size_t)c.width * c.height;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        r->anc_n = s->anc.n;
        r->bytes = footprint(s->cfg, (size_t)s->anc.n * s->cfg.k, r->nv, r->pixels);
        r->ticket = s->next_ticket++;
        r->t_submit = s->now_ms();
        s->reqs[r->ticket] = r;
        s->queue.push_back(r);
        *ticket = r->ticket;
    }
    s->cv.notify_all();
    return UPS_OK;
}

ups_status ups_poll(ups_server *s, uint64_t ticket, ups_result *out) {
    if (!s) return UPS_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return UPS_ERR_ARG;
    Req *r = it->second;
    if (out) {
        out->status = r->status;
        out->submit_ms = r->t_submit;
        out->start_ms = r->t_start;
        out->end_ms = r->t_end;
        out->batch_id = r->batch_id;
        out->batch_requests = r->batch_reqs;
        out->batch_views = r->batch_views;
    }
    if (r->status == UPS_PENDING) return UPS_PENDING;
    s->reqs.erase(it);
    delete r;
    return UPS_OK;
}

ups_status ups_cancel(ups_server *s, uint64_t ticket) {
    if (!s) return UPS_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return UPS_ERR_ARG;
    Req *r = it->second;
    if (r->started) return UPS_ERR_STATE;
    s->queue.erase(std::remove(s->queue.begin(), s->queue.end(), r), s->queue.end());
    r->status = UPS_ERR_CANCELLED;
    r->t_end = s->now_ms();
    return UPS_OK;
}

ups_status ups_server_wait_idle(ups_server *s, double timeout_ms) {
    if (!s) return UPS_ERR_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    bool ok = s->cv.wait_for(lk, std::chrono::duration<double, std::milli>(timeout_ms),
                             [&] { return s->queue.empty() && s->in_flight == 0; });
    return ok ? UPS_OK : UPS_ERR_TIMEOUT;
}

ups_status ups_server_set_scene(ups_server *s, const ups_anchors *scene, const ups_mlp *mlp, double timeout_ms) {
    if (!s || !scene || !mlp || scene->n < 1 || !scene->pos || !scene->feat || !scene->offsets || !scene->scaling ||
        !mlp->w1 || !mlp->b1 || !mlp->w2 || !mlp->b2)
        return UPS_ERR_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    s->paused = true;
    // in_flight drops when a batch's stream work has completed (host callback)
    const bool ok = s->cv.wait_for(lk, std::chrono::duration<double, std::milli>(timeout_ms),
                                   [&] { return s->in_flight == 0; });
    if (ok) {
        s->anc = *scene;
        s->mlp = *mlp;
        for (Req *r : s->queue) r->bytes = footprint(s->cfg, (size_t)s->anc.n * s->cfg.k, r->nv, r->pixels);
    }
    s->paused = false;
    lk.unlock();
    s->cv.notify_all();
    return ok ? UPS_OK : UPS_ERR_TIMEOUT;
}

const char *ups_server_last_error(const ups_server *s) { return s ? s->err.c_str() : ""; }

}  // extern "C"
