// lazy.cuh -- the fused-update gradient pass of plain (single-slab) volumes.
//
// One 3MG iteration of a volume that is not split into slabs is two passes:
//
//   k_gradlazy   applies the update of the previous iteration (Master box step
//                (2): x += D u, d = D u, and with them H d = -u0 H g + u1 H d,
//                r += H d) as it reads the state, then forms the gradient g of
//                the new iterate (Worker step (3)) and its objective f
//                (Section 3.1, Eq. "crit"; trace, stopping test);
//   k_curvature  H g, the inner products of D^T A D and D^T grad f (Eq. "maj")
//                and, in its last CTA, the 2x2 solve u = -B^+ c (Eq. "minimizer").
//
// so the separate update pass (40 B per voxel) and the objective pass (8 B) of
// the slab iteration disappear: the gradient pass reads x, g, d, r, H g, H d
// (24 B) and writes x, d, r, H d, g (20 B).  Because the pass reads r, H g, H d
// with a halo of the PSF radius and x, g, d with a halo of one voxel while it
// writes the same quantities, it reads one buffer set and writes the other;
// VolRun::par names the set holding a volume's current state and
// VolRun::pending whether the last solve's u still has to be applied.  Both
// are device words, flipped by the launches themselves, so one captured graph
// serves every iteration.  k_flush (update.cu) applies a pending update and
// brings the state back to set 0 before anything else reads it.
//
// The update arithmetic is the one of k_update (n = fmaf(-u0, g, u1 d),
// x + n; H n = fmaf(-u0, H g, u1 H d), r + H n), so the iterates are the bits
// the separate update pass produces.
#pragma once
#include "kernels.cuh"

namespace bd3mg {

// Shared memory of k_gradlazy: rings of PREF + 1 slices for r, H g and H d
// (r is combined into r + H n in place; with BF16 directions the H g and H d
// slots hold BF16 tiles of their own geometry, inside the same bytes), a ring
// of three slices of the updated
// iterate x + n over the tile and a one-voxel halo (rows -1 .. 32 of width
// XTW: column col at index col + 2, so the thread's column pair is 8-byte
// aligned), the x-pass output and the PSF rows.
template <int R, int RZ>
struct LazyGeo {
    using G = Geo<R, RZ, TY_A>;
    static constexpr int NS = PREF + 1;
    static constexpr int XTW = TX + 4, XTH = TY_A + 2, XTS = XTW * XTH;
    static constexpr int NHALO = 2 * (TX + 2) + 2 * TY_A;       // halo voxels of one slice
    static constexpr size_t SMEM =
        sizeof(float) * (3 * NS * G::SLOT + 3 * XTS + G::BY * TX + G::CF_FLOATS) + G::bars_bytes(NS);
    static_assert(NHALO <= NT, "one halo voxel per thread");
    static_assert((3 * XTS) % 4 == 0, "the x-pass output must stay 16-byte aligned");
};

// gradlazy_item processes work item `item` and returns false when a bounded
// wait ran out; k_gradlazy runs item blockIdx.x, the persistent iteration
// (PERS) every item a CTA takes from the pass's queue.
//
// BD (BD3MG_BF16_DIRECTIONS, with BF): d, H g and H d are stored as BF16.  Their
// staged tiles start 8 columns left of the tile (a TMA box of 16-bit elements
// must start on a 16-byte boundary), HOFF columns left of r's.
template <int R, int RZ, bool BF, int PM, bool PERS, bool BD = false>
__device__ __forceinline__ bool gradlazy_item(const KArgs &a, int item) {
    using G = Geo<R, RZ, TY_A>;
    using T = typename std::conditional<BF, __nv_bfloat16, float>::type;   // storage of g
    using DT = typename std::conditional<BD, __nv_bfloat16, float>::type;  // storage of d, H g, H d
    constexpr int KZ = G::KZ, NS = LazyGeo<R, RZ>::NS, BX = G::BX, BY = G::BY, SLOT = G::SLOT, XH = G::XH;
    // staged H g / H d tiles: halo XHB columns, width BXB, SLOTB elements per slot (128-byte multiple)
    constexpr int XHB = BD ? 8 : XH, BXB = TX + 2 * XHB, HOFF = XHB - XH;
    constexpr int SLOTB = BD ? ((BXB * BY * 2 + 127) / 128 * 128) / 2 : SLOT;
    static_assert(SLOTB * sizeof(DT) <= SLOT * sizeof(float), "the H g / H d slots must fit the FP32 layout");
    extern __shared__ __align__(128) float smem[];
    float *sr = smem;                                    // NS * SLOT: r, then r + H n in place
    DT *shg = reinterpret_cast<DT *>(sr + NS * SLOT);   // NS * SLOTB: H g
    DT *shd = shg + NS * SLOTB;                          // NS * SLOTB: H d
    using LG = LazyGeo<R, RZ>;
    constexpr int XTW = LG::XTW, XTS = LG::XTS;
    float *xt = sr + 3 * NS * SLOT;                      // 3 * XTS: x + n of slices z (slot (z - zo0 + 1) mod 3)
    float *T1 = xt + 3 * XTS;
    float *CF = T1 + BY * TX;
    uint64_t *bar = reinterpret_cast<uint64_t *>(CF + G::CF_FLOATS);

    const Item it = a.items[item];
    const unsigned long long wait_ns = a.sh->wait_ns;
    const SegDev sg = a.segs[it.seg];
    const VolDev &V = a.vols[sg.vol];
    const int nx = V.nx, ny = V.ny, nz = V.nz, pitch = V.pitch;
    const long long plane = V.plane;
    const float delta2 = V.delta2, xmin = V.xmin, xmax = V.xmax, lam = V.lam, eta2 = V.eta2, kap2 = V.kap2;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (vol_stopped(a, sg.vol)) {
        if (publish_zero<3>(a.partials, a.ticket, a.nitems, item)) objective_finish(a);
        return true;
    }
    // the volume's current buffer set, and whether the last solve's update is still to be applied
    const VolRun &rv = a.sh->run[sg.vol];
    const bool set1 = __ldcg(&rv.par) != 0;
    const bool apply = __ldcg(&rv.pending) != 0;
    float u0 = 0.f, u1 = 0.f;
    if (apply) {
        u0 = (float)a.u[2 * sg.slot];
        u1 = (float)a.u[2 * sg.slot + 1];
    }
    // source set (read) and destination set (written; the same when nothing is applied)
    const float *xs = set1 ? V.x1 : V.x;
    const DT *ds = reinterpret_cast<const DT *>(set1 ? V.d1 : V.d);
    const T *gs;
    T *gd;
    if constexpr (BF) {
        gs = set1 ? V.gh1 : V.gh;
        gd = (set1 != apply) ? V.gh1 : V.gh;
    } else {
        gs = set1 ? V.g1 : V.g;
        gd = (set1 != apply) ? V.g1 : V.g;
    }
    const bool dset1 = set1 != apply;
    float *xd = dset1 ? V.x1 : V.x, *rd = dset1 ? V.r1 : V.r;
    DT *dd = reinterpret_cast<DT *>(dset1 ? V.d1 : V.d);
    DT *hdd = reinterpret_cast<DT *>(dset1 ? sg.hd1 : sg.hd);

    const int zbeg = it.zo0 - RZ, zend = it.zo1 + RZ;
    stage_coeffs<G>(CF, V, zbeg, zend - zbeg);
    if (!init_bars(bar, NS, smem, a.sh->status)) return false;
    const int rlo = max(0, zbeg), rhi = min(nz, zend);
    const VolMaps &vm = a.maps[sg.vol];
    const CUtensorMap *mr = &vm.m[set1 ? TM_R1_R : TM_R_R];
    const CUtensorMap *mhg = &vm.m[set1 ? TM_HG1_R : TM_HG_R];
    const CUtensorMap *mhd = &vm.m[set1 ? TM_HD1_R : TM_HD_R];
    if (tid == 0) {
        asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(reinterpret_cast<uint64_t>(mr)) : "memory");
        if (apply) {
            asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(reinterpret_cast<uint64_t>(mhg)) : "memory");
            asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(reinterpret_cast<uint64_t>(mhd)) : "memory");
        }
    }
    const uint32_t nb = (uint32_t)(BX * BY * sizeof(float)), nbh = (uint32_t)(BXB * BY * sizeof(DT));
    const int bx0 = it.tx0 - XH, by0 = it.ty0 - R;
    // slice z of r (and of H g, H d when an update is applied) into ring slot s
    auto issue = [&](int z, int s) {
        if (tid == 0 && z >= rlo && z < rhi) {
            mbar_expect_tx(bar + s, apply ? nb + 2u * nbh : nb);
            tma_load_3d(sr + s * SLOT, mr, bx0, by0, z, bar + s);
            if (apply) {
                tma_load_3d(shg + s * SLOTB, mhg, it.tx0 - XHB, by0, z, bar + s);
                tma_load_3d(shd + s * SLOTB, mhd, it.tx0 - XHB, by0, z, bar + s);
            }
        }
    };
#pragma unroll
    for (int p = 0; p < PREF; ++p) issue(zbeg + p, p);
    __syncthreads();

    constexpr int XP = Units<G::XUNITS>::PER;
    int xsrc[XP], xdst[XP];
#pragma unroll
    for (int j = 0; j < XP; ++j) xpass_offsets<G>(tid + j * NT, xsrc[j], xdst[j]);
    const int yo = 4 * warp + 2 * (lane >> 4), c = 2 * (lane & 15);
    const int gx = it.tx0 + c, gy = it.ty0 + yo;
    const bool c0ok = gx < nx, c1ok = gx + 1 < nx, r0ok = gy < ny, r1ok = gy + 1 < ny;
    const bool own = r0ok && c0ok;
    const long long o0 = (long long)gy * pitch + gx, o1 = o0 + pitch;
    const int ci = (yo + R) * BX + XH + c;               // staged index of (yo, c)
    // ur0/ur1[t]: H_xy^T (r + H n) of the rows (yo, yo+1) x columns (c, c+1) for slice zi - ((S - t) mod KZ)
    float2 ur0[KZ], ur1[KZ];
#pragma unroll
    for (int t = 0; t < KZ; ++t) ur0[t] = ur1[t] = make_float2(0.f, 0.f);
    float acc[3] = {0.f, 0.f, 0.f};                      // data, box, penalty / lambda
    uint32_t par = 0u;
    bool timed_out = false;
    int zi = zbeg, sl = 0;

    // halo voxel of this thread in the iterate tile (threads < NHALO): its row and
    // column relative to the tile, and its index in a tile slice
    int hrow = 0, hcol = 0;
    if (tid < 2 * (TX + 2)) {
        hrow = tid < TX + 2 ? -1 : TY_A;
        hcol = (tid < TX + 2 ? tid : tid - (TX + 2)) - 1;
    } else if (tid < LG::NHALO) {
        const int t = tid - 2 * (TX + 2);
        hrow = t < TY_A ? t : t - TY_A;
        hcol = t < TY_A ? -1 : TX;
    }
    const int hgx = it.tx0 + hcol, hgy = it.ty0 + hrow;
    const bool hin = tid < LG::NHALO && hgx >= 0 && hgx < nx && hgy >= 0 && hgy < ny;
    const long long hoff = (long long)hgy * pitch + hgx;
    const int hidx = (hrow + 1) * XTW + hcol + 2;
    const int oidx = (yo + 1) * XTW + c + 2;             // index of (yo, c) in a tile slice
    auto xslot = [&](int z) { return xt + ((z - it.zo0 + 1) % 3) * XTS; };

    auto step = [&](auto sc) -> bool {
        constexpr int S = decltype(sc)::value;
        if (zi >= zend) return false;
        const int zo = zi - RZ;
        const bool emit = zo >= it.zo0;
        const bool ld = zi >= rlo && zi < rhi;
        const bool mine = zi >= it.zo0 && zi < it.zo1;   // the item's own depths for r and H d
        float *rs = sr + sl * SLOT;
        bool ok = true;
        if (ld) {
            ok = mbar_wait(bar + sl, (par >> sl) & 1u, wait_ns);
            if (ok) par ^= 1u << sl;
            if (ok && apply) {
                // r + H n over the staged tile, in place
                const DT *hgt = shg + sl * SLOTB, *hdt = shd + sl * SLOTB;
                float4 *r4 = reinterpret_cast<float4 *>(rs);
                for (int i = tid; i < BX * BY / 4; i += NT) {
                    float4 h, d;
                    if constexpr (BD) {
                        const int row = i / (BX / 4), e = row * BXB + 4 * (i - row * (BX / 4)) + HOFF;
                        const uint2 hq = *reinterpret_cast<const uint2 *>(hgt + e);
                        const uint2 dq = *reinterpret_cast<const uint2 *>(hdt + e);
                        const float2 h0 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&hq.x));
                        const float2 h1 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&hq.y));
                        const float2 d0 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&dq.x));
                        const float2 d1 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&dq.y));
                        h = make_float4(h0.x, h0.y, h1.x, h1.y);
                        d = make_float4(d0.x, d0.y, d1.x, d1.y);
                    } else {
                        h = reinterpret_cast<const float4 *>(hgt)[i];
                        d = reinterpret_cast<const float4 *>(hdt)[i];
                    }
                    float4 r = r4[i];
                    r.x += fmaf(-u0, h.x, u1 * d.x);
                    r.y += fmaf(-u0, h.y, u1 * d.y);
                    r.z += fmaf(-u0, h.z, u1 * d.z);
                    r.w += fmaf(-u0, h.w, u1 * d.w);
                    r4[i] = r;
                }
                // order these generic writes before the slot's next TMA write
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            }
        }
        if (__syncthreads_or(!ok)) {
            timed_out = true;
            return false;
        }
        issue(zi + PREF, sl + PREF >= NS ? sl + PREF - NS : sl + PREF);
        // slice zt = zo + 1 of the updated iterate x + n: its loads now, its tile
        // after the x-pass (slices zo0 - 1 .. zo1 are the penalty's z window)
        const int zt = zo + 1;
        const bool build = zt >= it.zo0 - 1 && zt <= it.zo1 && zt >= 0 && zt < nz;
        float2 bx[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)}, bg[2] = {bx[0], bx[0]}, bd[2] = {bx[0], bx[0]};
        float hxv = 0.f, hgv = 0.f, hdv = 0.f;
        if (build) {
            const long long zoff = (long long)zt * plane;
            if (own) {
                bx[0] = ldm<PERS>(reinterpret_cast<const float2 *>(xs + zoff + o0));
                if (r1ok) bx[1] = ldm<PERS>(reinterpret_cast<const float2 *>(xs + zoff + o1));
                if (apply) {
                    bg[0] = ld2(gs + zoff + o0);
                    bd[0] = ldp<PERS>(ds + zoff + o0);
                    if (r1ok) {
                        bg[1] = ld2(gs + zoff + o1);
                        bd[1] = ldp<PERS>(ds + zoff + o1);
                    }
                }
            }
            if (hin) {
                hxv = ldm<PERS>(xs + zoff + hoff);
                if (apply) {
                    hgv = to_f(gs[zoff + hoff]);
                    hdv = lds<PERS>(ds + zoff + hoff);
                }
            }
        }
        if (ld) {
            if (mine && own) {
                // r and H d of the item's own voxels at depth zi, and the data term 1/2 r^2
                const float2 ra = ld2(rs + ci), rb = ld2(rs + ci + BX);
                acc[0] = fmaf(0.5f * ra.x, ra.x, acc[0]);
                if (c1ok) acc[0] = fmaf(0.5f * ra.y, ra.y, acc[0]);
                if (r1ok) {
                    acc[0] = fmaf(0.5f * rb.x, rb.x, acc[0]);
                    if (c1ok) acc[0] = fmaf(0.5f * rb.y, rb.y, acc[0]);
                }
                if (apply) {
                    const int cih = (yo + R) * BXB + XHB + c;                 // staged index of (yo, c), H tiles
                    const DT *hgs = shg + sl * SLOTB + cih, *hds = shd + sl * SLOTB + cih;
                    const float2 ga = ld2(hgs), gb = ld2(hgs + BXB), da = ld2(hds), db = ld2(hds + BXB);
                    const float2 na = make_float2(fmaf(-u0, ga.x, u1 * da.x), fmaf(-u0, ga.y, u1 * da.y));
                    const float2 nb2 = make_float2(fmaf(-u0, gb.x, u1 * db.x), fmaf(-u0, gb.y, u1 * db.y));
                    const long long zoff = (long long)zi * plane;   // the zone of a whole volume starts at 0
                    if (c1ok) {
                        *reinterpret_cast<float2 *>(rd + zoff + o0) = ra;
                        stp(hdd + zoff + o0, na);
                        if (r1ok) {
                            *reinterpret_cast<float2 *>(rd + zoff + o1) = rb;
                            stp(hdd + zoff + o1, nb2);
                        }
                    } else {
                        rd[zoff + o0] = ra.x;
                        sts(hdd + zoff + o0, na.x);
                        if (r1ok) {
                            rd[zoff + o1] = rb.x;
                            sts(hdd + zoff + o1, nb2.x);
                        }
                    }
                }
            }
            const float *cfi = CF + (zi - zbeg) * G::CFS;
            float fxc[G::KXY];
            row_coeffs(fxc, cfi);
#pragma unroll
            for (int j = 0; j < XP; ++j)
                if (tid + j * NT < G::XUNITS) xpass_unit<G, R, +1>(rs, T1, xsrc[j], xdst[j], fxc);
        }
        if (build) {
            // x + n into the tile (zero outside the volume); with an applied update
            // the item's own depths also write x + n and n = D u to the destination set
            float *tz = xslot(zt);
            float2 xn[2], nn[2];
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                nn[k] = make_float2(fmaf(-u0, bg[k].x, u1 * bd[k].x), fmaf(-u0, bg[k].y, u1 * bd[k].y));
                xn[k] = apply ? make_float2(bx[k].x + nn[k].x, bx[k].y + nn[k].y) : bx[k];
            }
            *reinterpret_cast<float2 *>(tz + oidx) = own ? xn[0] : make_float2(0.f, 0.f);
            *reinterpret_cast<float2 *>(tz + oidx + XTW) = (own && r1ok) ? xn[1] : make_float2(0.f, 0.f);
            if (tid < LG::NHALO) tz[hidx] = hin ? (apply ? hxv + fmaf(-u0, hgv, u1 * hdv) : hxv) : 0.f;
            if (apply && own && zt >= it.zo0 && zt < it.zo1) {
                const long long zoff = (long long)zt * plane;
                if (c1ok) {
                    *reinterpret_cast<float2 *>(xd + zoff + o0) = xn[0];
                    stp(dd + zoff + o0, nn[0]);
                    if (r1ok) {
                        *reinterpret_cast<float2 *>(xd + zoff + o1) = xn[1];
                        stp(dd + zoff + o1, nn[1]);
                    }
                } else {
                    xd[zoff + o0] = xn[0].x;
                    sts(dd + zoff + o0, nn[0].x);
                    if (r1ok) {
                        xd[zoff + o1] = xn[1].x;
                        sts(dd + zoff + o1, nn[1].x);
                    }
                }
            }
        }
        __syncthreads();
        if (ld) {
            float fyc[G::KXY];
            row_coeffs(fyc, CF + (zi - zbeg) * G::CFS + G::KXYP);
            ypassT_pair2<R>(T1, yo, c, fyc, ur0[S], ur1[S]);
        } else {
            ur0[S] = ur1[S] = make_float2(0.f, 0.f);
        }
        if (emit) {
            // q(zo) = sum_t fz_{zo+t-RZ}[t] u(zo + t - RZ); u of slice zi - 2RZ + t in ring index (S + 1 + t) mod KZ
            float2 qa0 = make_float2(0.f, 0.f), qb0 = qa0, qa1 = qa0, qb1 = qa0;
#pragma unroll
            for (int t = 0; t < KZ; ++t) {
                const float f = CF[(zo + t - RZ - zbeg) * G::CFS + 2 * G::KXYP + t];
                const float2 f2 = make_float2(f, f);
                const int ri = (S + 1 + t) % KZ;
                if (t & 1) {
                    qb0 = __ffma2_rn(f2, ur0[ri], qb0);
                    qb1 = __ffma2_rn(f2, ur1[ri], qb1);
                } else {
                    qa0 = __ffma2_rn(f2, ur0[ri], qa0);
                    qa1 = __ffma2_rn(f2, ur1[ri], qa1);
                }
            }
            float2 q0 = __fadd2_rn(qa0, qb0), q1 = __fadd2_rn(qa1, qb1);
            if (own) {
                // the updated iterate around the block, from the tile ring
                const float *tm = xslot(zo - 1) + oidx, *tc = xslot(zo) + oidx, *tp = xslot(zo + 1) + oidx;
                auto X1 = [&](int dz, int dy, int dx) { return (dz < 0 ? tm : dz > 0 ? tp : tc)[dy * XTW + dx]; };
                auto X2 = [&](int dz, int dy, int dx) { return ld2((dz < 0 ? tm : dz > 0 ? tp : tc) + dy * XTW + dx); };
                const float2 p0 = X2(0, 0, 0);
                const float2 p1 = r1ok ? X2(0, 1, 0) : p0;
                const PenCtx pk{c1ok, r1ok, gx >= 1, gx + 2 < nx, gy >= 1, gy + 2 < ny, zo >= 1, zo + 1 < nz,
                                delta2, lam, eta2, kap2, V.kl, xmin, xmax};
                float ob[2] = {0.f, 0.f};
                pen_block<PM, true>(X1, X2, pk, p0, p1, q0, q1, ob);
                acc[1] += ob[0];
                acc[2] += ob[1];
                // g of the new iterate
                const long long zoff = (long long)zo * plane;
                if constexpr (BF) {
                    if (c1ok) *reinterpret_cast<__nv_bfloat162 *>(gd + zoff + o0) = __floats2bfloat162_rn(q0.x, q0.y);
                    else gd[zoff + o0] = __float2bfloat16_rn(q0.x);
                    if (r1ok) {
                        if (c1ok) *reinterpret_cast<__nv_bfloat162 *>(gd + zoff + o1) = __floats2bfloat162_rn(q1.x, q1.y);
                        else gd[zoff + o1] = __float2bfloat16_rn(q1.x);
                    }
                } else {
                    if (c1ok) *reinterpret_cast<float2 *>(gd + zoff + o0) = q0;
                    else gd[zoff + o0] = q0.x;
                    if (r1ok) {
                        if (c1ok) *reinterpret_cast<float2 *>(gd + zoff + o1) = q1;
                        else gd[zoff + o1] = q1.x;
                    }
                }
            }
        }
        ++zi;
        sl = sl + 1 == NS ? 0 : sl + 1;
        return true;
    };
    while (for_slots<0, KZ>(step)) {
    }
    if (timed_out) {
        if (tid == 0) {
            for (int z = zi; z < min(zi + PREF, zend + PREF); ++z) {
                if (z < rlo || z >= rhi) continue;
                const int s = (z - zbeg) % NS;
                if (mbar_wait(bar + s, (par >> s) & 1u, wait_ns)) par ^= 1u << s;
            }
            atomicOr(a.sh->status, ST_TIMEOUT);
        }
        return false;
    }
    item_end<PERS>(bar, NS);
    if (publish_partials<3>(acc, a.partials, a.ticket, a.nitems, item)) objective_finish(a);
    return true;
}

template <int R, int RZ, bool BF, int PM, bool BD = false>
__global__ void __launch_bounds__(NT, 2) k_gradlazy(KArgs a) {
    gradlazy_item<R, RZ, BF, PM, false, BD>(a, blockIdx.x);
}

}  // namespace bd3mg
