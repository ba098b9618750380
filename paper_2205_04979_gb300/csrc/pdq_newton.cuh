// pdq_newton.cuh -- the particle-particle Coulomb sums of Eq. coulomb (App. A.2: a direct
// sum within a sample, minimum image in z, the contact-distance clamp) with each unordered
// pair evaluated once (Newton pairs), packed FP32: the pair math, the z-range
// classification of tile pairs and the per-tile sum shared by the step (k_pairs_sym) and the
// adjoint's forward sweep.
#pragma once

#include <type_traits>

#include "pdq_device.cuh"

namespace pdq {

// ---------------------------------------------------------------------------
// The Coulomb sums with each unordered pair evaluated once
// (Newton's third law, G(-d) = -G(d)): a_i += q_j G(d) and a_j -= q_i G(d), d = x_i - x_j,
// G(d) = d / max(|d|, d_c)^3.  Per packed pair (two i-particles, one j) 16 f32x2
// operations and 2 rsqrt give four ordered pairs, against 12 and 2 for two ordered pairs
// in the one-sided loop.  MINIMG: per-pair minimum image in z (else the tile pair's uniform
// shift is folded into zi); CLAMP: some pair of the tiles may come closer than d_c.
// nqi = -q_i; the j-side sums of the two lanes land in (jx, jy, jz).
// ---------------------------------------------------------------------------
template <bool MINIMG, bool CLAMP>
__device__ __forceinline__ void coulomb_pair_x2_sym(f2 xi, f2 yi, f2 zi, f2 nqi, f2 xj, f2 yj, f2 zj, f2 qj,
                                                    f2 invL2, f2 M2, f2 nM2, f2 nL2, float c2, f2& ax, f2& ay,
                                                    f2& az, f2& jx, f2& jy, f2& jz) {
    const f2 dx = f2_sub(xi, xj), dy = f2_sub(yi, yj);
    f2 dz = f2_sub(zi, zj);
    if constexpr (MINIMG) {
        const f2 t = f2_add(f2_fma(dz, invL2, M2), nM2);
        dz = f2_fma(nL2, t, dz);
    }
    const f2 r2 = f2_fma(dx, dx, f2_fma(dy, dy, f2_mul(dz, dz)));
    float ra, rb;
    f2_unpack(r2, ra, rb);
    if constexpr (CLAMP) { ra = fmaxf(ra, c2); rb = fmaxf(rb, c2); }
    const f2 ri = f2_pack(rsqrt_ftz(ra), rsqrt_ftz(rb));
    const f2 ri3 = f2_mul(f2_mul(ri, ri), ri);
    const f2 si = f2_mul(ri3, qj), sj = f2_mul(ri3, nqi);
    ax = f2_fma(si, dx, ax);
    ay = f2_fma(si, dy, ay);
    az = f2_fma(si, dz, az);
    jx = f2_fma(sj, dx, jx);
    jy = f2_fma(sj, dy, jy);
    jz = f2_fma(sj, dz, jz);
}

// z-range classification of an i-range [alo, ahi] against a j-range [blo, bhi] (as in k_step):
// inside one period window the minimum image is a uniform shift; z-separated by more than
// dcz the clamp is dropped too.
struct ZClass { bool direct, apart; float shift; };
__device__ __forceinline__ ZClass zclass(float alo, float ahi, float blo, float bhi, float Lf, float dcz) {
    const float dlo = alo - bhi, dhi = ahi - blo, halfL = 0.5f * Lf;
    ZClass t{true, false, 0.f};
    if (dlo > -halfL && dhi < halfL) t.shift = 0.f;
    else if (dlo > halfL && dhi < 3.f * halfL) t.shift = Lf;
    else if (dhi < -halfL && dlo > -3.f * halfL) t.shift = -Lf;
    else t.direct = false;
    t.apart = t.direct && ((dlo - t.shift > dcz) || (dhi - t.shift < -dcz));
    return t;
}

// Coulomb sums of one i-tile: particles [base, base + NT*U) of a sample ending at `end`, paired
// with every particle of the sample from `base` on, added into acc (x, y, z; w untouched).
// Warp w holds the i-particles [32 U w, 32 U (w + 1)) of the tile (lane l: 32 k + l, k < U), a
// contiguous run of the z-binned sample, so its z range is narrow and more j groups are z-separated
// from it (no clamp, no per-pair minimum image: 1.2 % of the groups need them for a z-sorted sample,
// against 4 % with the particles strided over the tile).
// Newton pairs run as 32-j groups: lane l holds j = (l + k) mod 32 at step k and passes that j's
// running sum to lane l - 1 after the step, so that within a warp no two lanes touch the same j and
// after 32 steps every sum is back at its own lane.  The running sums stay packed (one half per
// i-half of the packed pairs) and move as 64-bit shuffles; the halves are added once, at home.
// Each staged 32-j group sits twice in a row, so lane l reads entry l + k without wrapping
// (constant offsets in the unrolled loop).
//   - The tile's own particles (the diagonal block), warp by warp with no CTA barrier: warp w's
//     block of 32 U particles one-sided against itself, and Newton pairs with the other warps'
//     blocks in a cyclic order that gives every warp the same number of pair evaluations (the
//     pass list is below).  A warp stages its j groups in its own slice of the staging arrays,
//     the next group's load in flight during a pass; the j-side sums are added in shared memory
//     and join the i-side sums at the end.  Of the block's pairs, 1/W run one-sided.
//   - The later particles: Newton pairs by j-tiles of NT staged by the whole CTA; the per-warp
//     j-side sums of a tile are added in shared memory and leave with one float4 atomic per j.
// The earlier particles of the sample reach this tile as the j side of earlier tiles.
// load(g) gives particle g as (x, y, z, q).  Padding particles sit far off the axis
// (x = +-1e15) with zero charge, so they add nothing.  All threads of the CTA take part; the
// shared arrays are the calling kernel's (one set per kernel instantiation).
template <int NT, int U, class Load>
__device__ __forceinline__ void newton_tile(const Load& load, int64_t base, int64_t end, float Lf, float invL,
                                            float c2, float4* __restrict__ acc) {
    constexpr int W = NT / 32, H = U / 2;
    static_assert(U % 4 == 0 && NT % 32 == 0, "packed pairs over whole warps, an even number of them");
    // the staged j particles pre-duplicated, (x,x,y,y) in sxy, (z,z,q,q) in szq and (z-L,z-L,q,q) in
    // szm (16-byte strides, so the skewed per-lane reads are free of bank conflicts), group r at
    // entries 64 r + t and 64 r + 32 + t; per-warp j-side sums of a j-tile; z range of each group;
    // the diagonal block's j-side sums
    __shared__ __align__(32) ulonglong2 sxy[2 * NT];
    __shared__ __align__(32) ulonglong2 szq[2 * NT];
    __shared__ __align__(32) ulonglong2 szm[2 * NT];
    __shared__ float s_jacc[W][3][NT];
    __shared__ float2 s_zr[W];
    __shared__ float s_dj[3][NT * U];
    // Register budget: the hot loop holds 7 H packed i-values and 4 H calls' temporaries, so
    // little else stays live across it: positions relative to `base` as 32-bit offsets (a
    // sample has fewer than 2^31 particles), no shifted copy of Z, and the minimum-image
    // constants built inside their (rare) branch.  A uniform z shift is exact either way:
    // shift -L takes the j side from szm (z_j - L is exact: such j have z_j > L/2, Sterbenz);
    // shift +L moves Z in place (z_i - L is exact for z_i > L/2, and adding L back restores z_i).
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const float dcz = sqrtf(c2) + 1e-3f;     // contact distance + rounding margin
    const float kPadI = 1e15f, kPadJ = -1e15f;
    const int n = (int)(end - base);                 // particles of the sample from base on
    const int nd = n < NT * U ? n : NT * U;          // the diagonal block
    for (int t = tid; t < 3 * NT * U; t += NT) (&s_dj[0][0])[t] = 0.f;
    f2 X[H], Y[H], Z[H], NQ[H], AX[H], AY[H], AZ[H];
    float ilo = INFINITY, ihi = -INFINITY;
#pragma unroll
    for (int h = 0; h < H; ++h) {
        float4 p[2];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int g = warp * (32 * U) + (2 * h + e) * 32 + lane;
            if (g < n) {
                p[e] = load(base + g);
                ilo = fminf(ilo, p[e].z);
                ihi = fmaxf(ihi, p[e].z);
            } else {
                p[e] = make_float4(kPadI, 0.f, 0.f, 0.f);
            }
        }
        X[h] = f2_pack(p[0].x, p[1].x);
        Y[h] = f2_pack(p[0].y, p[1].y);
        Z[h] = f2_pack(p[0].z, p[1].z);
        NQ[h] = f2_pack(-p[0].w, -p[1].w);
        AX[h] = AY[h] = AZ[h] = 0ull;
    }
    for (int d = 16; d > 0; d >>= 1) {     // this warp's i range
        ilo = fminf(ilo, __shfl_xor_sync(0xffffffffu, ilo, d));
        ihi = fmaxf(ihi, __shfl_xor_sync(0xffffffffu, ihi, d));
    }
    __syncthreads();                       // s_dj zeroed
    auto shift_z = [&](float sh) {
        const f2 s2 = f2_pack(sh, sh);
#pragma unroll
        for (int h = 0; h < H; ++h) Z[h] = f2_sub(Z[h], s2);
    };
    const float nLf = -Lf;
    const int from = (lane + 1) & 31;
    // Newton pairs of this warp's packed pairs h >= HLO with the 32-j group staged at entries
    // [64 r, 64 r + 64), z range zr.  The j-side sums come back at their own lanes.
    auto newton_group = [&](int r, float2 zr, auto hlo, f2& JX, f2& JY, f2& JZ) {
        const ZClass zc = zclass(ilo, ihi, zr.x, zr.y, Lf, dcz);
        JX = JY = JZ = 0ull;
        const ulonglong2 *pa = sxy + 64 * r + lane, *pb = (zc.direct && zc.shift < 0.f ? szm : szq) + 64 * r + lane;
        auto body = [&](auto minimg, auto clamp) {
            f2 invL2 = 0ull, M2 = 0ull, nM2 = 0ull, nL2 = 0ull;
            if constexpr (decltype(minimg)::value) {
                const float M = 12582912.0f;
                invL2 = f2_pack(invL, invL); M2 = f2_pack(M, M); nM2 = f2_pack(-M, -M); nL2 = f2_pack(-Lf, -Lf);
            }
#pragma unroll 4
            for (int k = 0; k < 32; ++k) {
                const ulonglong2 a = pa[k], b = pb[k];
#pragma unroll
                for (int h = decltype(hlo)::value; h < H; ++h)
                    coulomb_pair_x2_sym<decltype(minimg)::value, decltype(clamp)::value>(
                        X[h], Y[h], Z[h], NQ[h], a.x, a.y, b.x, b.y, invL2, M2, nM2, nL2, c2, AX[h], AY[h], AZ[h],
                        JX, JY, JZ);
                JX = __shfl_sync(0xffffffffu, JX, from);
                JY = __shfl_sync(0xffffffffu, JY, from);
                JZ = __shfl_sync(0xffffffffu, JZ, from);
            }
        };
        if (zc.direct) {
            const bool up = zc.shift > 0.f;
            if (up) shift_z(Lf);
            if (zc.apart && decltype(hlo)::value == 0) body(std::false_type{}, std::false_type{});
            else body(std::false_type{}, std::true_type{});
            if (up) shift_z(nLf);
        } else {
            body(std::true_type{}, std::true_type{});
        }
    };

    // ---- the diagonal block, warp by warp ----
    // Warp w's i-particles are block B_w (2H groups of 32).  Passes of warp w, one staged 32-j group
    // each: (0) the groups of B_w, one-sided; (1) the groups of B_{w+d}, d = 1 .. (W-1)/2, Newton
    // pairs; for W even, B_w and B_{w+W/2} once: warp w < W/2 takes the first H groups of
    // B_{w+W/2} with all its packed pairs, warp w >= W/2 the 2H groups of B_{w-W/2} with its
    // packed pairs h >= H/2 (the last H groups of B_w).  Every warp issues the same number of pair
    // evaluations; within a pass all its packed pairs take part.
    {
        constexpr int DN = (W - 1) / 2, NP0 = 2 * H, NP1 = NP0 + 2 * H * DN;
        constexpr int NPW = NP1 + ((W % 2 == 0) ? 2 * H : 0);
        const int ngd = (nd + 31) >> 5;                                   // 32-groups with particles
        const int ival = nd - warp * 32 * U;                              // this warp's i-particles (if > 0)
        // pass t -> its j group (or -1: nothing to do) and kind
        auto pass_of = [&](int t, int& kind) -> int {
            int G;
            if (t < NP0) { kind = 0; G = 2 * H * warp + t; }
            else if (t < NP1) { kind = 1; const int d = 1 + (t - NP0) / (2 * H); G = 2 * H * ((warp + d) % W) + (t - NP0) % (2 * H); }
            else if (warp < W / 2) { kind = 1; const int u = t - NP1; G = u < H ? 2 * H * (warp + W / 2) + u : -1; }
            else { kind = 2; G = 2 * H * (warp - W / 2) + (t - NP1); }
            const bool has_i = kind == 2 ? ival > 32 * H : ival > 0;
            return (G >= 0 && G < ngd && has_i) ? G : -1;
        };
        auto fetch = [&](int G) {
            const int jj = 32 * G + lane;
            return (G >= 0 && jj < nd) ? load(base + jj) : make_float4(kPadJ, 0.f, 0.f, 0.f);
        };
        int kind;
        int G = pass_of(0, kind);
        float4 pj = fetch(G);
#pragma unroll 1
        for (int t = 0; t < NPW; ++t) {
            int kind_n;
            const int Gn = t + 1 < NPW ? pass_of(t + 1, kind_n) : -1;
            const float4 pn = fetch(Gn);                                  // the next pass's j, in flight
            if (G >= 0) {
                const bool real = 32 * G + lane < nd;
                float jlo = real ? pj.z : INFINITY, jhi = real ? pj.z : -INFINITY;
                for (int d = 16; d > 0; d >>= 1) {
                    jlo = fminf(jlo, __shfl_xor_sync(0xffffffffu, jlo, d));
                    jhi = fmaxf(jhi, __shfl_xor_sync(0xffffffffu, jhi, d));
                }
                {
                    const ulonglong2 vxy = make_ulonglong2(f2_pack(pj.x, pj.x), f2_pack(pj.y, pj.y));
                    const ulonglong2 vzq = make_ulonglong2(f2_pack(pj.z, pj.z), f2_pack(pj.w, pj.w));
                    const float zm = pj.z + nLf;
                    const ulonglong2 vzm = make_ulonglong2(f2_pack(zm, zm), f2_pack(pj.w, pj.w));
                    const int e = warp * 64 + lane;
                    __syncwarp();                      // the slice's previous group is no longer read
                    sxy[e] = vxy; sxy[e + 32] = vxy;
                    szq[e] = vzq; szq[e + 32] = vzq;
                    szm[e] = vzm; szm[e + 32] = vzm;
                    __syncwarp();
                }
                const float2 zr = make_float2(jlo, jhi);
                if (kind == 0) {
                    // one-sided, every i of the warp with every j of the group (the self pair adds nothing)
                    const ZClass zc = zclass(ilo, ihi, zr.x, zr.y, Lf, dcz);
                    float mn = 0.f;
                    if (zc.direct) {
                        const bool up = zc.shift > 0.f;
                        if (up) shift_z(Lf);
                        const ulonglong2 *pa = sxy + 64 * warp, *pb = (zc.shift < 0.f ? szm : szq) + 64 * warp;
#pragma unroll 4
                        for (int k = 0; k < 32; ++k) {
                            const ulonglong2 a = pa[k], b = pb[k];
#pragma unroll
                            for (int h = 0; h < H; ++h)
                                coulomb_pair_x2_direct<true>(X[h], Y[h], Z[h], a.x, a.y, b.x, b.y, c2, AX[h], AY[h],
                                                             AZ[h], mn);
                        }
                        if (up) shift_z(nLf);
                    } else {
                        const float M = 12582912.0f;
                        const f2 invL2 = f2_pack(invL, invL), M2 = f2_pack(M, M), nM2 = f2_pack(-M, -M);
                        const f2 nL2 = f2_pack(-Lf, -Lf);
                        const ulonglong2 *pa = sxy + 64 * warp, *pb = szq + 64 * warp;
#pragma unroll 4
                        for (int k = 0; k < 32; ++k) {
                            const ulonglong2 a = pa[k], b = pb[k];
#pragma unroll
                            for (int h = 0; h < H; ++h)
                                coulomb_pair_x2<false>(X[h], Y[h], Z[h], a.x, a.y, b.x, b.y, invL2, M2, nM2, nL2, c2,
                                                       AX[h], AY[h], AZ[h], mn);
                        }
                    }
                } else {
                    f2 JX, JY, JZ;
                    if (kind == 1) newton_group(warp, zr, std::integral_constant<int, 0>{}, JX, JY, JZ);
                    else newton_group(warp, zr, std::integral_constant<int, H / 2>{}, JX, JY, JZ);
                    float l0, l1;
                    f2_unpack(JX, l0, l1); atomicAdd(&s_dj[0][32 * G + lane], l0 + l1);
                    f2_unpack(JY, l0, l1); atomicAdd(&s_dj[1][32 * G + lane], l0 + l1);
                    f2_unpack(JZ, l0, l1); atomicAdd(&s_dj[2][32 * G + lane], l0 + l1);
                }
            }
            G = Gn; kind = kind_n; pj = pn;
        }
        __syncthreads();                       // every warp's slice free, s_dj complete
    }

    // ---- Newton pairs with the later particles, by j-tiles of NT (the next tile's particle in
    // flight during a tile) ----
    float4 pj = nd + tid < n ? load(base + nd + tid) : make_float4(kPadJ, 0.f, 0.f, 0.f);
    for (int j0 = nd; j0 < n; j0 += NT) {
        const int j = j0 + tid;
        float jlo = j < n ? pj.z : INFINITY, jhi = j < n ? pj.z : -INFINITY;
        for (int d = 16; d > 0; d >>= 1) {
            jlo = fminf(jlo, __shfl_xor_sync(0xffffffffu, jlo, d));
            jhi = fmaxf(jhi, __shfl_xor_sync(0xffffffffu, jhi, d));
        }
        if (lane == 0) s_zr[warp] = make_float2(jlo, jhi);
        {
            const ulonglong2 vxy = make_ulonglong2(f2_pack(pj.x, pj.x), f2_pack(pj.y, pj.y));
            const ulonglong2 vzq = make_ulonglong2(f2_pack(pj.z, pj.z), f2_pack(pj.w, pj.w));
            const float zm = pj.z + nLf;
            const ulonglong2 vzm = make_ulonglong2(f2_pack(zm, zm), f2_pack(pj.w, pj.w));
            const int e = warp * 64 + lane;
            sxy[e] = vxy; sxy[e + 32] = vxy;
            szq[e] = vzq; szq[e + 32] = vzq;
            szm[e] = vzm; szm[e + 32] = vzm;
        }
        __syncthreads();
        const float4 pnext = j + NT < n ? load(base + j + NT) : make_float4(kPadJ, 0.f, 0.f, 0.f);
#pragma unroll 1
        for (int g = 0; g < W; ++g) {
            f2 JX, JY, JZ;
            newton_group(g, s_zr[g], std::integral_constant<int, 0>{}, JX, JY, JZ);
            float l0, l1;
            f2_unpack(JX, l0, l1); s_jacc[warp][0][g * 32 + lane] = l0 + l1;
            f2_unpack(JY, l0, l1); s_jacc[warp][1][g * 32 + lane] = l0 + l1;
            f2_unpack(JZ, l0, l1); s_jacc[warp][2][g * 32 + lane] = l0 + l1;
        }
        __syncthreads();
        if (j < n) {
            float sx = 0.f, sy = 0.f, sz = 0.f;
#pragma unroll
            for (int w = 0; w < W; ++w) { sx += s_jacc[w][0][tid]; sy += s_jacc[w][1][tid]; sz += s_jacc[w][2][tid]; }
            atomicAdd(&acc[base + j], make_float4(sx, sy, sz, 0.f));
        }
        pj = pnext;
    }
#pragma unroll
    for (int h = 0; h < H; ++h) {
        float a0[3], a1[3];
        f2_unpack(AX[h], a0[0], a1[0]);
        f2_unpack(AY[h], a0[1], a1[1]);
        f2_unpack(AZ[h], a0[2], a1[2]);
        const int g0 = warp * (32 * U) + (2 * h) * 32 + lane, g1 = g0 + 32;
        if (g0 < n) atomicAdd(&acc[base + g0], make_float4(a0[0] + s_dj[0][g0], a0[1] + s_dj[1][g0], a0[2] + s_dj[2][g0], 0.f));
        if (g1 < n) atomicAdd(&acc[base + g1], make_float4(a1[0] + s_dj[0][g1], a1[1] + s_dj[1][g1], a1[2] + s_dj[2][g1], 0.f));
    }
}

}  // namespace pdq
