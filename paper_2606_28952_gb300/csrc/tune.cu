// tune.cu -- the autotuner of the apply launch shape: columns per thread,
// staged source rows in flight, piece-range splits per row and direct vs
// staged gather are timed on the device for one (operator, sector, dtype) and
// the fastest is kept in the operator's plan for that sector.
#include <algorithm>
#include <cfloat>
#include <cstdio>
#include <cstdlib>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "ps_internal.cuh"

using namespace ps;

namespace {

constexpr int kTuneMaxCandidates = 96;

void store_tuned(Plan &p, const SectorView &v, int dtype, const LaunchChoice &c, double ms) {
    for (TunedEntry &t : p.tuned)
        if (t.dim == v.dim && t.nblk == v.nblk && t.dtype == dtype) {
            t.choice = c;
            t.ms = ms;
            return;
        }
    p.tuned.push_back(TunedEntry{v.dim, v.nblk, dtype, c, ms});
}

void ensure_split_capacity(pauli_sum *H, Plan &p, int64_t bytes) {
    if (p.split_cap >= bytes) return;
    PS_CUDA(cudaDeviceSynchronize());
    dev_free(H->al, p.split_buf);
    p.split_buf = nullptr;
    p.split_cap = 0;
    p.split_buf = dev_alloc(H->al, (size_t)bytes);
    p.split_cap = bytes;
}

pauli_launch_config to_public(const ApplyCfg &c, double ms) {
    pauli_launch_config o;
    o.cols_per_thread = c.tpt;
    o.staged_rows = c.nbuf;
    o.row_split = c.nsplit;
    o.direct = c.svd ? 4 : (c.list ? 3 : (c.local ? 2 : (c.direct ? 1 : 0)));
    o.ranked = c.ranked ? 1 : 0;
    o.ms = ms;
    return o;
}


// Cache key of (H, s) on the current device: the device name, the sector's
// shape, the operator's sizes and a 64-bit FNV-1a fingerprint of its canonical
// arrays (x, z, C), so that a cached shape is only installed on the operator and
// sector it was measured for.
std::string tune_key(const pauli_sum *H, const pauli_sector *s) {
    int dev = 0;
    PS_CUDA(cudaGetDevice(&dev));
    cudaDeviceProp prop;
    PS_CUDA(cudaGetDeviceProperties(&prop, dev));
    std::string name(prop.name);
    for (char &ch : name)
        if (ch == ' ' || ch == '|' || ch == '\t') ch = '_';
    uint64_t fp = 1469598103934665603ull;
    auto mix = [&](const void *p, size_t bytes) {
        const unsigned char *b = static_cast<const unsigned char *>(p);
        for (size_t i = 0; i < bytes; ++i) {
            fp ^= b[i];
            fp *= 1099511628211ull;
        }
    };
    if (H->m > 0) {
        std::vector<uint64_t> hx(H->m), hz(H->m);
        std::vector<double2> hc(H->m);
        PS_CUDA(cudaMemcpy(hx.data(), H->x, H->m * 8, cudaMemcpyDeviceToHost));
        PS_CUDA(cudaMemcpy(hz.data(), H->z, H->m * 8, cudaMemcpyDeviceToHost));
        PS_CUDA(cudaMemcpy(hc.data(), H->c, H->m * 16, cudaMemcpyDeviceToHost));
        mix(hx.data(), hx.size() * 8);
        mix(hz.data(), hz.size() * 8);
        mix(hc.data(), hc.size() * 16);
    }
    const SectorView &v = s->v;
    std::ostringstream k;
    k << name << "|n" << v.n << "|lo" << v.n_lo << "|k" << v.kind << "|b";
    if (v.kind == PAULI_SECTOR_BLOCKS)
        for (int b = 0; b < v.nblk; ++b) k << (b ? "," : "") << v.klo[b] << ":" << v.khi[b];
    char hex[17];
    std::snprintf(hex, sizeof(hex), "%016llx", (unsigned long long)fp);
    k << "|d" << v.dim << "|M" << H->m << "|G" << H->G << "|" << hex;
    return k.str();
}

constexpr const char *kTuneTag = "paulisim-tune-v1";

}  // namespace

extern "C" {

int pauli_tune(pauli_sum *H, const pauli_sector *s, int dtype, int reps, pauli_launch_config *best,
               pauli_stream_t st) {
    try {
        clear_error();
        PS_CHECK(H && H->magic == kSumMagic, PAULI_EINVAL, "not a valid pauli_sum handle");
        PS_CHECK(s && s->magic == kSectorMagic, PAULI_EINVAL, "not a valid pauli_sector handle");
        PS_CHECK(H->n == s->v.n, PAULI_EINVAL, "operator and sector have different qubit counts");
        PS_CHECK(dtype == PAULI_C64 || dtype == PAULI_C128, PAULI_EINVAL, "bad dtype");
        PS_CHECK(reps >= 1 && reps <= 1000, PAULI_EINVAL, "reps must be in 1..1000");
        cudaStream_t cs = (cudaStream_t)st;
        Plan &p = get_plan(H, s->v, cs);
        const SectorView &v = s->v;
        prepare_for_sector(H, p, v, cs);
        // candidates
        std::vector<LaunchChoice> cand;
        const bool fits = p.I <= 256 && p.S <= 1024;
        if (s->v.kind == PAULI_SECTOR_FULL)
            for (int cl : {0, 1})
                for (int tpt : {4, 8}) {
                    if (!(cl ? p.local_cl : p.local)) continue;
                    LaunchChoice c;
                    c.direct = 2;
                    c.ranked = cl;
                    c.tpt = tpt;
                    cand.push_back(c);
                }
        if (v.kind == PAULI_SECTOR_BLOCKS && v.nblk == 1 && find_lists(p, v.klo[0]))
            for (int ns : {1, 2, 4, 8, 16}) {
                if (ns > 1 && ns > std::max<int64_t>(1, p.P / 8)) continue;
                LaunchChoice c;
                c.direct = 3;
                c.nsplit = ns;
                const ApplyCfg cfg = apply_config(p, v, dtype, true, &c);
                if (!cfg.list || cfg.nsplit != ns || cfg.smem > 226 * 1024) continue;
                cand.push_back(c);
            }
        if (v.kind == PAULI_SECTOR_BLOCKS && v.nblk == 1 && H->real) {
            if (!svd_plan_fits(p.svd, v)) {
                free_svd_plan(p.svd);
                p.svd = nullptr;
                p.svd = build_svd_plan(H, v, cs);
            }
            if (p.svd && svd_batches(p.svd) <= 4)
                for (int tpt : {1, 2, 4}) {
                    LaunchChoice c;
                    c.tpt = tpt;
                    c.direct = 4;
                    if (apply_config(p, v, dtype, true, &c).svd && svd_smem(v, dtype) <= 226 * 1024) cand.push_back(c);
                }
        }
        for (int tpt : {1, 2, 4, 8}) {
            if (fits && tpt < 8) {
                LaunchChoice c;
                c.tpt = tpt;
                c.direct = 1;
                cand.push_back(c);
            }
            for (int ranked : {0, 1})
                for (int nbuf : {1, 2})
                    for (int ns : {1, 2, 4, 8, 16}) {
                        if (ns > 1 && ns > std::max<int64_t>(1, p.P / 8)) continue;
                        LaunchChoice c;
                        c.tpt = tpt;
                        c.nbuf = nbuf;
                        c.nsplit = ns;
                        c.direct = 0;
                        c.ranked = ranked;
                        const ApplyCfg cfg = apply_config(p, v, dtype, true, &c);
                        // not realisable, or the layout does not fit in shared memory
                        if (cfg.nbuf != nbuf || cfg.nsplit != ns || (int)cfg.ranked != ranked || cfg.tpt != tpt)
                            continue;
                        if (tpt == 8 && nbuf != 1) continue;
                        if (cfg.smem > 226 * 1024) continue;
                        cand.push_back(c);
                    }
        }
        // at most kTuneMaxCandidates shapes are timed (in the order enumerated above)
        if ((int)cand.size() > kTuneMaxCandidates) cand.resize(kTuneMaxCandidates);
        // scratch states and the largest split buffer any candidate needs
        const size_t es = dtype == PAULI_C64 ? 8 : 16;
        int64_t need = 0;
        for (const LaunchChoice &c : cand) need = std::max(need, apply_split_elems(p, v, dtype, &c) * (int64_t)es);
        ensure_split_capacity(H, p, need);
        if (dtype == PAULI_C128)
            for (const LaunchChoice &c : cand)
                if (c.direct == 3) {
                    ensure_df_buffer(H, p, v, cs);
                    break;
                }
        DevBuf<char> in(H->al, (size_t)v.dim * es), out(H->al, (size_t)v.dim * es);
        PS_CUDA(cudaMemsetAsync(in.p, 0x3c, (size_t)v.dim * es, cs));
        cudaEvent_t e0, e1;
        PS_CUDA(cudaEventCreate(&e0));
        PS_CUDA(cudaEventCreate(&e1));
        double best_ms = DBL_MAX;
        LaunchChoice best_c;
        ApplyCfg best_cfg;
        try {
            for (const LaunchChoice &c : cand) {
                launch_apply(H, p, v, in.p, out.p, dtype, nullptr, cs, true, &c);  // warm-up
                PS_CUDA(cudaEventRecord(e0, cs));
                for (int r = 0; r < reps; ++r) launch_apply(H, p, v, in.p, out.p, dtype, nullptr, cs, true, &c);
                PS_CUDA(cudaEventRecord(e1, cs));
                PS_CUDA(cudaEventSynchronize(e1));
                float ms = 0.f;
                PS_CUDA(cudaEventElapsedTime(&ms, e0, e1));
                const double per = ms / reps;
                if (per < best_ms) {
                    best_ms = per;
                    best_c = c;
                    best_cfg = apply_config(p, v, dtype, true, &c);
                }
            }
        } catch (...) {
            (void)cudaEventDestroy(e0);
            (void)cudaEventDestroy(e1);
            throw;
        }
        (void)cudaEventDestroy(e0);
        (void)cudaEventDestroy(e1);
        PS_CUDA(cudaStreamSynchronize(cs));
        store_tuned(p, v, dtype, best_c, best_ms);
        if (best) *best = to_public(best_cfg, best_ms);
        return PAULI_OK;
    } catch (const Error &e) {
        set_error(e.msg);
        return e.code;
    } catch (...) {
        set_error("unexpected internal error");
        return PAULI_EINVAL;
    }
}

int pauli_set_launch_config(pauli_sum *H, const pauli_sector *s, int dtype, const pauli_launch_config *cfg) {
    try {
        clear_error();
        PS_CHECK(H && H->magic == kSumMagic, PAULI_EINVAL, "not a valid pauli_sum handle");
        PS_CHECK(s && s->magic == kSectorMagic, PAULI_EINVAL, "not a valid pauli_sector handle");
        PS_CHECK(H->n == s->v.n, PAULI_EINVAL, "operator and sector have different qubit counts");
        PS_CHECK(dtype == PAULI_C64 || dtype == PAULI_C128, PAULI_EINVAL, "bad dtype");
        PS_CHECK(cfg != nullptr, PAULI_EINVAL, "cfg is NULL");
        PS_CHECK(cfg->cols_per_thread == 1 || cfg->cols_per_thread == 2 || cfg->cols_per_thread == 4 ||
                     cfg->cols_per_thread == 8,
                 PAULI_EINVAL, "cols_per_thread must be 1, 2, 4 or 8");
        PS_CHECK(cfg->staged_rows == 1 || cfg->staged_rows == 2, PAULI_EINVAL, "staged_rows must be 1 or 2");
        PS_CHECK(cfg->row_split >= 1 && cfg->row_split <= 16, PAULI_EINVAL, "row_split must be in 1..16");
        PS_CHECK(cfg->direct >= 0 && cfg->direct <= 4, PAULI_EINVAL, "direct must be 0, 1, 2, 3 or 4");
        PS_CHECK(cfg->ranked == 0 || cfg->ranked == 1, PAULI_EINVAL, "ranked must be 0 or 1");
        cudaStream_t cs = nullptr;
        PS_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        try {
            Plan &p = get_plan(H, s->v, cs);
            prepare_for_sector(H, p, s->v, cs);
            if (cfg->direct == 4) {
                if (!svd_plan_fits(p.svd, s->v)) {
                    free_svd_plan(p.svd);
                    p.svd = nullptr;
                    p.svd = build_svd_plan(H, s->v, cs);
                }
                PS_CHECK(p.svd != nullptr, PAULI_EUNSUPPORTED,
                         "the SVD gather needs a real operator on a single product block with a low half of at "
                         "most 16 qubits");
            }
            LaunchChoice c;
            c.tpt = cfg->cols_per_thread;
            c.nbuf = cfg->staged_rows;
            c.nsplit = cfg->row_split;
            c.direct = cfg->direct;
            c.ranked = cfg->ranked;
            const size_t es = dtype == PAULI_C64 ? 8 : 16;
            ensure_split_capacity(H, p, apply_split_elems(p, s->v, dtype, &c) * (int64_t)es);
            store_tuned(p, s->v, dtype, c, cfg->ms);
            ensure_df_capacity(H, p, s->v, cs);
        } catch (...) {
            (void)cudaStreamDestroy(cs);
            throw;
        }
        PS_CUDA(cudaStreamSynchronize(cs));
        (void)cudaStreamDestroy(cs);
        return PAULI_OK;
    } catch (const Error &e) {
        set_error(e.msg);
        return e.code;
    } catch (...) {
        set_error("unexpected internal error");
        return PAULI_EINVAL;
    }
}

int pauli_get_launch_config(pauli_sum *H, const pauli_sector *s, int dtype, pauli_launch_config *cfg) {
    try {
        clear_error();
        PS_CHECK(H && H->magic == kSumMagic, PAULI_EINVAL, "not a valid pauli_sum handle");
        PS_CHECK(s && s->magic == kSectorMagic, PAULI_EINVAL, "not a valid pauli_sector handle");
        PS_CHECK(dtype == PAULI_C64 || dtype == PAULI_C128, PAULI_EINVAL, "bad dtype");
        PS_CHECK(cfg != nullptr, PAULI_EINVAL, "cfg is NULL");
        Plan *p = find_plan(H, s->v);
        PS_CHECK(p != nullptr, PAULI_EINVAL, "no plan for this sector split yet: call pauli_prepare first");
        double ms = 0.0;
        for (const TunedEntry &t : p->tuned)
            if (t.dim == s->v.dim && t.nblk == s->v.nblk && t.dtype == dtype) ms = t.ms;
        *cfg = to_public(apply_config(*p, s->v, dtype, true), ms);
        return PAULI_OK;
    } catch (const Error &e) {
        set_error(e.msg);
        return e.code;
    }
}

int pauli_tune_save(pauli_sum *H, const pauli_sector *s, const char *path) {
    try {
        clear_error();
        PS_CHECK(H && H->magic == kSumMagic, PAULI_EINVAL, "not a valid pauli_sum handle");
        PS_CHECK(s && s->magic == kSectorMagic, PAULI_EINVAL, "not a valid pauli_sector handle");
        PS_CHECK(path != nullptr && *path, PAULI_EINVAL, "path is NULL or empty");
        Plan *p = find_plan(H, s->v);
        PS_CHECK(p != nullptr, PAULI_EINVAL, "no plan for this sector split yet: call pauli_prepare first");
        const std::string key = tune_key(H, s);
        std::vector<std::string> keep;
        {
            std::ifstream in(path);
            std::string line;
            while (std::getline(in, line)) {
                std::istringstream ls(line);
                std::string tag, k, dt;
                if (!(ls >> tag >> k >> dt) || tag != kTuneTag) continue;
                bool replaced = false;
                for (const TunedEntry &t : p->tuned)
                    if (t.dim == s->v.dim && t.nblk == s->v.nblk && k == key &&
                        dt == (t.dtype == PAULI_C64 ? "c64" : "c128"))
                        replaced = true;
                if (!replaced) keep.push_back(line);
            }
        }
        int wrote = 0;
        for (const TunedEntry &t : p->tuned) {
            if (t.dim != s->v.dim || t.nblk != s->v.nblk) continue;
            std::ostringstream ls;
            ls.precision(17);
            ls << kTuneTag << " " << key << " " << (t.dtype == PAULI_C64 ? "c64" : "c128") << " " << t.choice.tpt << " "
               << t.choice.nbuf << " " << t.choice.nsplit << " " << t.choice.direct << " " << t.choice.ranked << " "
               << t.ms;
            keep.push_back(ls.str());
            ++wrote;
        }
        const std::string tmp = std::string(path) + ".tmp";
        {
            std::ofstream out(tmp, std::ios::trunc);
            PS_CHECK(out.good(), PAULI_EINVAL, std::string("cannot write ") + tmp);
            for (const std::string &l : keep) out << l << "\n";
            out.flush();
            PS_CHECK(out.good(), PAULI_EINVAL, std::string("write to ") + tmp + " failed");
        }
        PS_CHECK(std::rename(tmp.c_str(), path) == 0, PAULI_EINVAL, std::string("cannot replace ") + path);
        (void)wrote;
        return PAULI_OK;
    } catch (const Error &e) {
        set_error(e.msg);
        return e.code;
    } catch (...) {
        set_error("unexpected internal error");
        return PAULI_EINVAL;
    }
}

int pauli_tune_load(pauli_sum *H, const pauli_sector *s, const char *path, int *found) {
    try {
        clear_error();
        PS_CHECK(H && H->magic == kSumMagic, PAULI_EINVAL, "not a valid pauli_sum handle");
        PS_CHECK(s && s->magic == kSectorMagic, PAULI_EINVAL, "not a valid pauli_sector handle");
        PS_CHECK(H->n == s->v.n, PAULI_EINVAL, "operator and sector have different qubit counts");
        PS_CHECK(path != nullptr && *path, PAULI_EINVAL, "path is NULL or empty");
        PS_CHECK(found != nullptr, PAULI_EINVAL, "found is NULL");
        *found = 0;
        std::ifstream in(path);
        if (!in.good()) return PAULI_OK;  // no cache yet
        const std::string key = tune_key(H, s);
        std::string line;
        std::vector<std::pair<int, pauli_launch_config>> hits;
        while (std::getline(in, line)) {
            std::istringstream ls(line);
            std::string tag, k, dt;
            pauli_launch_config c;
            if (!(ls >> tag >> k >> dt >> c.cols_per_thread >> c.staged_rows >> c.row_split >> c.direct >> c.ranked >>
                  c.ms))
                continue;
            if (tag != kTuneTag || k != key || (dt != "c64" && dt != "c128")) continue;
            hits.emplace_back(dt == "c64" ? PAULI_C64 : PAULI_C128, c);
        }
        for (const auto &h : hits) {
            const int rc = pauli_set_launch_config(H, s, h.first, &h.second);
            if (rc != PAULI_OK) return rc;
            ++*found;
        }
        return PAULI_OK;
    } catch (const Error &e) {
        set_error(e.msg);
        return e.code;
    } catch (...) {
        set_error("unexpected internal error");
        return PAULI_EINVAL;
    }
}

int pauli_svd_ranks(pauli_sum *H, const pauli_sector *s, int *hist, int len, int *batches) {
    try {
        clear_error();
        PS_CHECK(H && H->magic == kSumMagic, PAULI_EINVAL, "not a valid pauli_sum handle");
        PS_CHECK(s && s->magic == kSectorMagic, PAULI_EINVAL, "not a valid pauli_sector handle");
        PS_CHECK(H->n == s->v.n, PAULI_EINVAL, "operator and sector have different qubit counts");
        PS_CHECK(hist != nullptr && len >= 1, PAULI_EINVAL, "hist is NULL or len < 1");
        cudaStream_t cs = nullptr;
        PS_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        try {
            Plan &p = get_plan(H, s->v, cs);
            if (!svd_plan_fits(p.svd, s->v)) {
                free_svd_plan(p.svd);
                p.svd = nullptr;
                p.svd = build_svd_plan(H, s->v, cs);
            }
            PS_CHECK(p.svd != nullptr, PAULI_EUNSUPPORTED,
                     "the SVD factorisation needs a real operator on a single product block (low half <= 16 qubits)");
            const std::vector<int> &h = svd_rank_hist(p.svd);
            for (int i = 0; i < len; ++i) hist[i] = i < (int)h.size() ? h[i] : 0;
            if (batches) *batches = svd_batches(p.svd);
        } catch (...) {
            (void)cudaStreamDestroy(cs);
            throw;
        }
        PS_CUDA(cudaStreamSynchronize(cs));
        (void)cudaStreamDestroy(cs);
        return PAULI_OK;
    } catch (const Error &e) {
        set_error(e.msg);
        return e.code;
    } catch (...) {
        set_error("unexpected internal error");
        return PAULI_EINVAL;
    }
}

}  // extern "C"
