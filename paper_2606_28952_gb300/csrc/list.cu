// list.cu -- the gather of eq. reverse_sum over lists of valid pairs, for
// single-block sectors whose low half has at most kListMaxLo qubits.
//
// In a single-block sector every row has the same low-half particle number
// k_lo, so whether the source t_lo ^ x_lo of a target t_lo lies in the block
// depends on x_lo and t_lo alone (Sec. 2.4: X flips occupations; the sector
// keeps only strings of the right popcount).  For a number-conserving
// molecular operator about half of the (item, target) pairs of a row fall
// outside: an X mask with two low bits set moves a particle only where
// exactly one of the two orbitals is occupied.  The staged gather computes
// those pairs and multiplies them by a zero slot.  Here every distinct x_lo of
// the plan gets, once per (plan, k_lo), the list of its valid pairs
// (rank of t_lo, rank of t_lo ^ x_lo, t_lo).  A CTA owns one row (all D_lo
// targets) and a range of its pieces; per piece it stages the source row
// densely by rank and folds the high-half phases into one coefficient per
// segment (as the staged gather does), then deals (item, chunk of the item's
// list) units round-robin to its warps.  A warp adds its units into its own
// accumulator row in shared memory: within a unit the targets are distinct,
// no two warps share a row, so there are no atomics, and the epilogue adds the
// warp rows in a fixed order.
#include <algorithm>
#include <unordered_map>
#include <vector>

#include "apply_kernels.cuh"

namespace ps {

namespace {

// 128-thread CTAs: four warp accumulator rows, so that two CTAs fit on an SM
// even in complex128 and one CTA's staging overlaps the other's gather
constexpr int kListThreads = 128;
constexpr int kListWarps = kListThreads / 32;
constexpr int kListK = 4;                     // list entries per lane in one unit
constexpr int kListChunk = 32 * kListK;       // entries of one unit
// the double-float path is latency-bound at two CTAs per SM (shared memory),
// with registers to spare: twice the independent entries per lane
constexpr int kListKDF = 8;
constexpr int kListChunkDF = 32 * kListKDF;
constexpr int kListTile = (int)kListMaxDlo;   // column tile of the geometry: a whole row

struct ListDev {
    const uint32_t *ent;
    const int32_t *off;
    const int32_t *it_list;
};

__host__ __device__ inline int list_row_pad(int64_t dlo) { return (int)((dlo + 1) & ~1ll); }

template <typename R>
__host__ __device__ inline size_t list_smem_r(int64_t dlo) {
    using C2 = typename Cx<R>::T;
    // warp accumulator rows, then one staging buffer (dense row by rank), then
    // the list range of each item of the piece
    return (size_t)kListWarps * list_row_pad(dlo) * sizeof(C2) + Smem<R>::buf_bytes(ranked_rowcap(dlo)) +
           (size_t)kItemCap * sizeof(int2);
}

// One unit: entries [base, base + kListChunk) of an item's list (those below
// len), lane-strided.  my: this warp's accumulator row.
template <typename R, bool REALH>
__device__ __forceinline__ void list_unit(const Buf<R> &B, const int4 e, const uint32_t *__restrict__ ent, int len,
                                          int base, int lane, typename Cx<R>::T *my) {
    using C2 = typename Cx<R>::T;
    uint32_t w[kListK];
    bool ok[kListK];
#pragma unroll
    for (int k = 0; k < kListK; ++k) {
        const int i = base + lane + 32 * k;
        ok[k] = i < len;
        w[k] = ok[k] ? __ldg(ent + i) : 0u;
    }
    uint32_t s[kListK];
    C2 amp[kListK];
    R fr[kListK], fi[kListK];
#pragma unroll
    for (int k = 0; k < kListK; ++k) {
        s[k] = (w[k] >> 20) ^ (uint32_t)e.x;
        amp[k] = B.row[(w[k] >> 10) & 1023u];
        fr[k] = R(0);
        fi[k] = R(0);
    }
    if (sizeof(R) == 4 && e.w) {
        // x = 0 group: compensated FP32 summation of the hi / lo coefficient pairs
        R er[kListK], ei[kListK];
#pragma unroll
        for (int k = 0; k < kListK; ++k) {
            er[k] = R(0);
            ei[k] = R(0);
        }
        for (int sg = e.y; sg < e.z; ++sg) {
            const uint32_t z = B.z[sg];
            const C2 a = B.a[sg];
            const float2 l = B.alo[sg];
#pragma unroll
            for (int k = 0; k < kListK; ++k) {
                const uint32_t par = __popc(z & s[k]);
                float t, err;
                two_sum(fr[k], flip((float)a.x, par), t, err);
                fr[k] = t;
                er[k] += err + flip(l.x, par);
                if (!REALH) {
                    two_sum(fi[k], flip((float)a.y, par), t, err);
                    fi[k] = t;
                    ei[k] += err + flip(l.y, par);
                }
            }
        }
#pragma unroll
        for (int k = 0; k < kListK; ++k) {
            fr[k] += er[k];
            fi[k] += ei[k];
        }
    } else {
        for (int sg = e.y; sg < e.z; ++sg) {
            const uint32_t z = B.z[sg];
            const C2 a = B.a[sg];
#pragma unroll
            for (int k = 0; k < kListK; ++k) {
                const uint32_t par = __popc(z & s[k]);
                fr[k] += flip(a.x, par);
                if (!REALH) fi[k] += flip(a.y, par);
            }
        }
    }
#pragma unroll
    for (int k = 0; k < kListK; ++k) {
        if (!ok[k]) continue;
        C2 &o = my[w[k] & 1023u];
        C2 t = o;
        if (REALH) {
            t.x += fr[k] * amp[k].x;
            t.y += fr[k] * amp[k].y;
        } else {
            t.x += fr[k] * amp[k].x - fi[k] * amp[k].y;
            t.y += fr[k] * amp[k].y + fi[k] * amp[k].x;
        }
        o = t;
    }
}

// ---------------------------------------------------------------------------
// complex128 in double-float arithmetic.  FP64 runs at a small fraction of the
// FP32 rate on this GPU, and the segment sums and accumulations of the gather
// are its inner loop.  The complex128 path therefore reads psi as hi + lo
// FP32 pairs (split once per apply by k_split_df: hi = fl32(v), lo =
// fl32(v - hi), 48 significant bits), keeps the folded segment coefficients
// and the accumulators as hi + lo pairs, and sums with Knuth's TwoSum and
// products split exactly with FMA (Dekker); the fold of the high-half phases
// and the epilogue stay FP64.
// ---------------------------------------------------------------------------
__global__ void k_split_df(const double2 *__restrict__ v, float4 *__restrict__ out, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double2 a = v[i];
    const float hr = __double2float_rn(a.x), hi = __double2float_rn(a.y);
    out[i] = make_float4(hr, hi, __double2float_rn(a.x - (double)hr), __double2float_rn(a.y - (double)hi));
}

// (ph, pl) = (fh + fl) * (ah + al) to about 2^-47 relative: the product of the
// high parts split exactly by FMA, plus the two cross terms (fl * al dropped)
__device__ __forceinline__ void df_mul(float fh, float fl, float ah, float al, float &ph, float &pl) {
    ph = __fmul_rn(fh, ah);
    const float e = __fmaf_rn(fh, ah, -ph);
    pl = __fmaf_rn(fh, al, __fmaf_rn(fl, ah, e));
}

// (h, l) += (ph, pl), renormalised so that |l| <= ulp(h) / 2
__device__ __forceinline__ void df_add(float &h, float &l, float ph, float pl) {
    float s, e;
    two_sum(h, ph, s, e);
    const float t = __fadd_rn(__fadd_rn(l, pl), e);
    const float hh = __fadd_rn(s, t);
    l = __fsub_rn(t, __fsub_rn(hh, s));
    h = hh;
}

// list_unit of the complex128 path: row and segment coefficients as float4
// {re hi, im hi, re lo, im lo}, accumulator row likewise.
template <bool REALH>
__device__ __forceinline__ void list_unit_df(const float4 *__restrict__ row, const float4 *__restrict__ a4,
                                             const uint32_t *__restrict__ zs, const int4 e,
                                             const uint32_t *__restrict__ ent, int len, int base, int lane,
                                             float4 *my) {
    uint32_t w[kListKDF];
    bool ok[kListKDF];
#pragma unroll
    for (int k = 0; k < kListKDF; ++k) {
        const int i = base + lane + 32 * k;
        ok[k] = i < len;
        w[k] = ok[k] ? __ldg(ent + i) : 0u;
    }
    uint32_t s[kListKDF];
    float4 amp[kListKDF];
    float frh[kListKDF], frl[kListKDF], fih[kListKDF], fil[kListKDF];
#pragma unroll
    for (int k = 0; k < kListKDF; ++k) {
        s[k] = (w[k] >> 20) ^ (uint32_t)e.x;
        amp[k] = row[(w[k] >> 10) & 1023u];
        frh[k] = frl[k] = fih[k] = fil[k] = 0.f;
    }
    // f = sum over the item's segments of +-a_seg: TwoSum on the high parts, the
    // rounding errors and the low parts summed beside them
    for (int sg = e.y; sg < e.z; ++sg) {
        const uint32_t z = zs[sg];
        const float4 a = a4[sg];
#pragma unroll
        for (int k = 0; k < kListKDF; ++k) {
            const uint32_t par = __popc(z & s[k]);
            float t, err;
            two_sum(frh[k], flip(a.x, par), t, err);
            frh[k] = t;
            frl[k] = __fadd_rn(frl[k], __fadd_rn(err, flip(a.z, par)));
            if (!REALH) {
                two_sum(fih[k], flip(a.y, par), t, err);
                fih[k] = t;
                fil[k] = __fadd_rn(fil[k], __fadd_rn(err, flip(a.w, par)));
            }
        }
    }
#pragma unroll
    for (int k = 0; k < kListKDF; ++k) {
        if (!ok[k]) continue;
        float4 &o = my[w[k] & 1023u];
        float4 t = o;
        float ph, pl;
        df_mul(frh[k], frl[k], amp[k].x, amp[k].z, ph, pl);  // f_re a_re
        df_add(t.x, t.z, ph, pl);
        df_mul(frh[k], frl[k], amp[k].y, amp[k].w, ph, pl);  // f_re a_im
        df_add(t.y, t.w, ph, pl);
        if (!REALH) {
            df_mul(fih[k], fil[k], amp[k].y, amp[k].w, ph, pl);  // - f_im a_im
            df_add(t.x, t.z, -ph, -pl);
            df_mul(fih[k], fil[k], amp[k].x, amp[k].z, ph, pl);  // + f_im a_re
            df_add(t.y, t.w, ph, pl);
        }
        o = t;
    }
}

template <typename R, bool REALH, bool DF>
__global__ void __launch_bounds__(kListThreads)
k_apply_list(SectorView v, Geom geo, PlanDev p, ListDev L, const typename Cx<R>::T *__restrict__ psi,
             const float4 *__restrict__ psi_df, typename Cx<R>::T *__restrict__ out, double *__restrict__ partials,
             int flags) {
    using C2 = typename Cx<R>::T;
    extern __shared__ __align__(16) char smem[];
    const int64_t dlo = v.dlo[0];
    const int dpad = list_row_pad(dlo);
    const int rw = ranked_rowcap(dlo);
    C2 *acc = reinterpret_cast<C2 *>(smem);
    char *bbase = smem + (size_t)kListWarps * dpad * sizeof(C2);
    Buf<R> B(bbase, rw);
    int2 *rng = reinterpret_cast<int2 *>(bbase + Smem<R>::buf_bytes(rw));
    const RowCtx rc = decode_row<false>(v, geo, blockIdx.x);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    {
        C2 zz;
        zz.x = R(0);
        zz.y = R(0);
        for (int i = tid; i < kListWarps * dpad; i += kListThreads) acc[i] = zz;
    }
    C2 *my = acc + (size_t)warp * dpad;
    int unused = 0;
    const int pend = geo.split_p0[rc.split + 1];
    int q = next_piece<R, KBLKR>(v, p, geo.split_p0[rc.split] - 1, rc.thi, pend);
    // the double-float path stages rows of the hi / lo split of psi (16 bytes per
    // amplitude, like complex128)
    const C2 *src = DF ? reinterpret_cast<const C2 *>(psi_df) : psi;
    while (q < pend) {
        stage_piece<R, KBLKR, REALH>(v, p, q, rc.thi, src, B, &unused);
        const int i0 = __ldg(p.pc_i0 + q), i1 = __ldg(p.pc_i0 + q + 1);
        for (int it = i0 + tid; it < i1; it += kListThreads) {
            const int l = __ldg(L.it_list + it);
            const int a = __ldg(L.off + l);
            rng[it - i0] = make_int2(a, __ldg(L.off + l + 1) - a);
        }
        cp_async_wait<0>();
        __syncthreads();
        if (DF) {
            // the folded FP64 segment coefficients -> hi / lo FP32 pairs, in place
            const int nseg = __ldg(p.it_s0 + i1) - __ldg(p.it_s0 + i0);
            float4 *a4 = reinterpret_cast<float4 *>(B.a);
            for (int sg = tid; sg < nseg; sg += kListThreads) {
                const C2 a = B.a[sg];
                const float hr = (float)a.x, hi = (float)a.y;
                a4[sg] = make_float4(hr, hi, (float)(a.x - (double)hr), (float)(a.y - (double)hi));
            }
            __syncthreads();
        }
        // unit u = (item, chunk) in item order goes to warp u mod kListWarps
        int u = 0;
        const int nit = i1 - i0;
        constexpr int kChunk = DF ? kListChunkDF : kListChunk;
        for (int it = 0; it < nit; ++it) {
            const int2 r = rng[it];
            const int nch = (r.y + kChunk - 1) / kChunk;
            int c = (warp - u) % kListWarps;
            if (c < 0) c += kListWarps;
            if (c < nch) {
                const int4 e = B.item[it];
                for (; c < nch; c += kListWarps) {
                    if constexpr (DF)
                        list_unit_df<REALH>(reinterpret_cast<const float4 *>(B.row),
                                            reinterpret_cast<const float4 *>(B.a), B.z, e, L.ent + r.x, r.y,
                                            c * kChunk, lane, reinterpret_cast<float4 *>(my));
                    else
                        list_unit<R, REALH>(B, e, L.ent + r.x, r.y, c * kListChunk, lane, my);
                    __syncwarp();
                }
            }
            u += nch;
        }
        __syncthreads();
        q = next_piece<R, KBLKR>(v, p, q, rc.thi, pend);
    }
    __syncthreads();

    // epilogue: the warp rows added in a fixed order; store and / or FP64 reductions
    ExpAcc<R> ea;
    for (int c = tid; c < dlo; c += kListThreads) {
        R sr = R(0), si = R(0);
        if constexpr (DF) {
            const float4 *acc4 = reinterpret_cast<const float4 *>(acc);
#pragma unroll
            for (int w = 0; w < kListWarps; ++w) {
                const float4 a = acc4[(size_t)w * dpad + c];
                sr += (double)a.x + (double)a.z;
                si += (double)a.y + (double)a.w;
            }
        } else {
#pragma unroll
            for (int w = 0; w < kListWarps; ++w) {
                const C2 a = acc[(size_t)w * dpad + c];
                sr += a.x;
                si += a.y;
            }
        }
        const int64_t idx = rc.own_base + c;
        if (flags & 1) {
            C2 o;
            o.x = sr;
            o.y = si;
            out[(flags & 4) ? (int64_t)rc.split * v.dim + idx : idx] = o;
        }
        if (flags & 2) ea.add(psi[idx], sr, si);
    }
    if (flags & 2) {
        double er = ea.get(0), ei = ea.get(1), h2 = ea.get(2), p2 = ea.get(3);
        __shared__ double red[4][kListWarps];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            er += __shfl_down_sync(0xffffffffu, er, o);
            ei += __shfl_down_sync(0xffffffffu, ei, o);
            h2 += __shfl_down_sync(0xffffffffu, h2, o);
            p2 += __shfl_down_sync(0xffffffffu, p2, o);
        }
        if (lane == 0) {
            red[0][warp] = er;
            red[1][warp] = ei;
            red[2][warp] = h2;
            red[3][warp] = p2;
        }
        __syncthreads();
        if (tid < 4) {
            double sum = 0.0;
            for (int w = 0; w < kListWarps; ++w) sum += red[tid][w];
            partials[(int64_t)blockIdx.x * 4 + tid] = sum;
        }
    }
}

template <typename R, bool REALH>
void launch_list_k(const ApplyCfg &cfg, const SectorView &v, const Geom &geo, const PlanDev &pd, const ListDev &ld,
                   const void *in, const float4 *in_df, void *out, double *partials, int flags, cudaStream_t st) {
    using C2 = typename Cx<R>::T;
    auto run = [&](auto kern) {
        smem_optin(reinterpret_cast<const void *>(kern), cfg.smem);
        kern<<<(unsigned)cfg.nct, kListThreads, cfg.smem, st>>>(v, geo, pd, ld, static_cast<const C2 *>(in), in_df,
                                                             static_cast<C2 *>(out), partials, flags);
        PS_LAUNCH_CHECK();
    };
    if constexpr (sizeof(R) == 8) {
        if (in_df) {
            run(k_apply_list<R, REALH, true>);
            return;
        }
    }
    run(k_apply_list<R, REALH, false>);
}

template <typename R>
void launch_list_r(const ApplyCfg &cfg, const Plan &p, const ListTab &lt, const SectorView &v, const void *in,
                   void *out, double *partials, void *split_buf, cudaStream_t st) {
    using C2 = typename Cx<R>::T;
    const Geom geo = make_geom(v, kListTile, cfg.nsplit, cfg.split_p0.data(), (int32_t)p.P);
    const PlanDev pd = plan_dev(p);
    ListDev ld;
    ld.ent = lt.ent;
    ld.off = lt.off;
    ld.it_list = lt.it_list;
    void *kout = out;
    int flags = (out ? 1 : 0) | (partials ? 2 : 0);
    if (cfg.nsplit > 1) {
        kout = split_buf;
        flags = 1 | 4;
    }
    const float4 *in_df = nullptr;
    if (sizeof(R) == 8) {
        // complex128: split psi into hi / lo FP32 pairs once, into the plan's buffer
        PS_CHECK(p.df_buf != nullptr && p.df_cap >= v.dim, PAULI_EINVAL,
                 "apply: the plan's double-float buffer is missing (internal)");
        if (v.dim > 0) {
            k_split_df<<<(unsigned)((v.dim + 255) / 256), 256, 0, st>>>(static_cast<const double2 *>(in), p.df_buf,
                                                                      v.dim);
            PS_LAUNCH_CHECK();
        }
        in_df = p.df_buf;
    }
    if (p.real) launch_list_k<R, true>(cfg, v, geo, pd, ld, in, in_df, kout, partials, flags, st);
    else launch_list_k<R, false>(cfg, v, geo, pd, ld, in, in_df, kout, partials, flags, st);
    if (cfg.nsplit > 1) {
        const int cflags = (out ? 1 : 0) | (partials ? 2 : 0);
        k_combine<R><<<(unsigned)cfg.combine_nct, kThreads, 0, st>>>(
            cfg.nsplit, v.dim, static_cast<const C2 *>(split_buf), static_cast<const C2 *>(in), static_cast<C2 *>(out),
            partials, cflags);
        PS_LAUNCH_CHECK();
    }
}

// The lists of one k_lo (host construction from the sector's own rank order).
void build_lists(const Allocator &al, Plan &p, const SectorView &v, cudaStream_t st) {
    const int n_lo = v.n_lo, klo = v.klo[0];
    const int64_t dlo = v.dlo[0];
    std::vector<uint32_t> pat(dlo > 0 ? dlo : 1);
    if (dlo > 0)
        PS_CUDA(cudaMemcpyAsync(pat.data(), v.list_lo + v.lst_lo_off[0], dlo * sizeof(uint32_t),
                                cudaMemcpyDeviceToHost, st));
    PS_CUDA(cudaStreamSynchronize(st));
    std::vector<int32_t> rank(1u << n_lo, -1);
    for (int64_t r = 0; r < dlo; ++r) rank[pat[r]] = (int32_t)r;
    std::unordered_map<uint32_t, int32_t> id;
    std::vector<uint32_t> ent;
    std::vector<int32_t> off(1, 0), it_list(p.I > 0 ? p.I : 1, 0), len;
    for (int64_t it = 0; it < p.I; ++it) {
        const uint32_t x = p.h_it_xlo[it];
        auto f = id.find(x);
        if (f == id.end()) {
            const int32_t l = (int32_t)(off.size() - 1);
            for (int64_t r = 0; r < dlo; ++r) {
                const int32_t sr = rank[pat[r] ^ x];
                if (sr >= 0) ent.push_back((uint32_t)r | ((uint32_t)sr << 10) | (pat[r] << 20));
            }
            off.push_back((int32_t)ent.size());
            len.push_back(off[l + 1] - off[l]);
            f = id.emplace(x, l).first;
        }
        it_list[it] = f->second;
    }
    ListTab &lt = p.lists[p.nlists];
    lt = ListTab();
    lt.klo = klo;
    lt.n_list = (int64_t)off.size() - 1;
    lt.n_ent = (int64_t)ent.size();
    auto upload = [&](const void *src, size_t bytes) {
        void *d = dev_alloc(al, bytes > 0 ? bytes : 4);
        if (bytes > 0) PS_CUDA(cudaMemcpy(d, src, bytes, cudaMemcpyHostToDevice));
        return d;
    };
    lt.ent = static_cast<uint32_t *>(upload(ent.data(), ent.size() * sizeof(uint32_t)));
    lt.off = static_cast<int32_t *>(upload(off.data(), off.size() * sizeof(int32_t)));
    lt.it_list = static_cast<int32_t *>(upload(it_list.data(), (size_t)p.I * sizeof(int32_t)));
    // work of a piece for its row: staging, plus per item its list chunks times
    // (one gather and accumulate per entry, one parity-add per segment and entry)
    lt.h_pc_cumw.assign(p.P + 1, 0);
    for (int64_t q = 0; q < p.P; ++q) {
        int64_t wq = 4 * dlo;
        for (int32_t it = p.h_pc_i0[q]; it < p.h_pc_i0[q + 1]; ++it) {
            const int64_t chunks = (len[it_list[it]] + kListChunk - 1) / kListChunk;
            wq += chunks * kListChunk * (6 + (p.h_it_s0[it + 1] - p.h_it_s0[it]));
        }
        lt.h_pc_cumw[q + 1] = lt.h_pc_cumw[q] + wq;
    }
    ++p.nlists;
}

}  // namespace

size_t list_smem(int dtype, int64_t dlo) {
    return dtype == PAULI_C64 ? list_smem_r<float>(dlo) : list_smem_r<double>(dlo);
}

const ListTab *find_lists(const Plan &p, int klo) {
    for (int i = 0; i < p.nlists; ++i)
        if (p.lists[i].klo == klo) return &p.lists[i];
    return nullptr;
}

void free_lists(const Allocator &al, Plan &p) {
    for (int i = 0; i < p.nlists; ++i) {
        dev_free(al, p.lists[i].ent);
        dev_free(al, p.lists[i].off);
        dev_free(al, p.lists[i].it_list);
        p.lists[i] = ListTab();
    }
    p.nlists = 0;
}

void prepare_for_sector(pauli_sum *H, Plan &p, const SectorView &v, cudaStream_t st) {
    if (v.kind == PAULI_SECTOR_FULL && !p.local_tried) {
        p.local_tried = true;
        p.local = build_local_plan(H, v.n, false, st);
        p.local_cl = build_local_plan(H, v.n, true, st);
    }
    if (v.kind == PAULI_SECTOR_BLOCKS && v.nblk == 1 && v.n_lo <= kListMaxLo && v.dlo[0] <= kListMaxDlo &&
        p.I > 0 && !find_lists(p, v.klo[0])) {
        if (p.nlists == kListCache) {  // drop the oldest
            PS_CUDA(cudaStreamSynchronize(st));
            dev_free(H->al, p.lists[0].ent);
            dev_free(H->al, p.lists[0].off);
            dev_free(H->al, p.lists[0].it_list);
            for (int i = 1; i < kListCache; ++i) p.lists[i - 1] = std::move(p.lists[i]);
            p.lists[kListCache - 1] = ListTab();
            p.nlists = kListCache - 1;
        }
        build_lists(H->al, p, v, st);
    }
}

void ensure_df_buffer(pauli_sum *H, Plan &p, const SectorView &v, cudaStream_t st) {
    if (p.df_cap >= v.dim) return;
    PS_CUDA(cudaStreamSynchronize(st));
    dev_free(H->al, p.df_buf);
    p.df_buf = nullptr;
    p.df_cap = 0;
    p.df_buf = static_cast<float4 *>(dev_alloc(H->al, (size_t)std::max<int64_t>(1, v.dim) * sizeof(float4)));
    p.df_cap = v.dim;
}

void ensure_df_capacity(pauli_sum *H, Plan &p, const SectorView &v, cudaStream_t st) {
    if (!find_lists(p, v.klo[0]) || !apply_config(p, v, PAULI_C128, true).list) return;
    ensure_df_buffer(H, p, v, st);
}

void launch_list(const ApplyCfg &cfg, const Plan &p, const SectorView &v, const void *in, void *out, int dtype,
                 double *partials, void *split_buf, cudaStream_t st) {
    const ListTab *lt = find_lists(p, v.klo[0]);
    PS_CHECK(lt != nullptr, PAULI_EINVAL, "apply: the pair lists of this sector are missing (internal)");
    if (dtype == PAULI_C64) launch_list_r<float>(cfg, p, *lt, v, in, out, partials, split_buf, st);
    else launch_list_r<double>(cfg, p, *lt, v, in, out, partials, split_buf, st);
}

}  // namespace ps
