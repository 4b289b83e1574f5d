// Slab-group step kernel (mixed precision).  One CTA per tile of zones, the
// tile's gas stencil staged in shared memory.  Inside a warp, three lanes own
// one sort key (one zone): lane a holds, in registers, the gas of the nine
// stencil nodes at x-offset a - 1 and the deposit accumulators of those nine
// nodes.  The three lanes push the zone's grains three at a time; weights,
// partial gathers and deposit impulses are exchanged with warp shuffles, so
// each grain's 27-node gather and deposit cost registers, not shared memory.
// A zone's deposit (its run: the grains sorted into it whose half-step host is
// the zone itself) is quantised once per node and flushed to the shared
// deposit box; the host node receives the remainder of the run's quantised
// total.  Grains stored in id order inside a zone (see the sort) make the
// summation order, hence the integers, reproducible.  Grains whose host is not
// their key zone (stale sort) use the per-grain rule.
//
// The push runs relative to the key zone: each coordinate's offset from the
// zone centre is formed once in double precision and rounded to single;
// the half drifts, the weights, the metric factors and the kick then work on
// these offsets in single precision, and the coordinate is updated once, in
// double precision, by the step's summed increment.  This keeps the narrow
// double-precision pipe to four operations per coordinate.
#pragma once

#include "dust_tiled.cuh"

namespace dust {

constexpr int kSlabThreads = 256;

template <int FLAT>
struct SlabShape {
    // FLAT: 0 = three gridded directions, 1 = y not gridded, 2 = z not gridded
    static constexpr int NB = FLAT == 1 ? 1 : 3;
    static constexpr int NC = FLAT == 2 ? 1 : 3;
    static constexpr int BC = NB == 3 ? 1 : 0;   // index of the host node in y
    static constexpr int CC = NC == 3 ? 1 : 0;   // index of the host node in z
};

__device__ __forceinline__ float sel3(const float v[3], int i)
{
    return i == 0 ? v[0] : (i == 1 ? v[1] : v[2]);
}

template <int GEOM, int FLAT>
__global__ void __launch_bounds__(kSlabThreads, 1)
step_slab_kernel(const TiledArgs<float> TA)
{
    using Sh = SlabShape<FLAT>;
    constexpr int NB = Sh::NB, NC = Sh::NC;
    const StepArgs<float> &A = TA.s;
    const GridDev &g = A.g;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const unsigned FULL = 0xffffffffu;

    const int tile = blockIdx.x;
    const int64_t kbase = (int64_t)tile * g.tvol;
    if (TA.key_off[kbase + g.tvol] <= TA.key_off[kbase]) return;

    int B[3], o[3], tc[3];
    tc[0] = tile % g.nt[0];
    tc[1] = (tile / g.nt[0]) % g.nt[1];
    tc[2] = tile / (g.nt[0] * g.nt[1]);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const int H = g.n[d] > 1 ? 1 : 0;
        B[d] = g.T[d] + 2 * H;
        o[d] = tc[d] * g.T[d] - H;
    }
    const int bvol = B[0] * B[1] * B[2];
    unsigned long long *sdep = reinterpret_cast<unsigned long long *>(smem_raw);
    float *sgas = reinterpret_cast<float *>(smem_raw + (size_t)bvol * 4 * sizeof(long long));

    for (int lin = threadIdx.x; lin < bvol; lin += blockDim.x) {
        const int bx = lin % B[0], by = (lin / B[0]) % B[1], bz = lin / (B[0] * B[1]);
        const int i = map_zone(o[0] + bx, g.n[0], g.bc[0]);
        const int j = map_zone(o[1] + by, g.n[1], g.bc[1]);
        const int k = map_zone(o[2] + bz, g.n[2], g.bc[2]);
        float v[4];
        load_gas<float>(A.gas, i + (int64_t)g.n[0] * (j + (int64_t)g.n[1] * k), v);
        smem_gas_store<float>(sgas, lin, v);
#pragma unroll
        for (int c = 0; c < 4; ++c) sdep[c * bvol + lin] = 0ull;
    }
    __syncthreads();

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int a = lane % 3, kq = lane / 3;
    const int base = lane - a;
    const int src1 = base + (a + 1) % 3, src2 = base + (a + 2) % 3;
    const float h = (float)(0.5 * A.dt), dt = (float)A.dt;
    const int groups = (g.tvol + 9) / 10;
    int nremoved = 0;
    float moved = 0.f;
    bool big = false;

    for (int grp = warp; grp < groups; grp += nwarps) {
        const int kl = grp * 10 + kq;
        const bool kok = lane < 30 && kl < g.tvol;
        int64_t off0 = 0;
        int cnt = 0;
        if (kok) {
            off0 = TA.key_off[kbase + kl];
            cnt = (int)(TA.key_off[kbase + kl + 1] - off0);
        }
        const int maxcnt = (int)__reduce_max_sync(FULL, (unsigned)cnt);
        if (maxcnt == 0) continue;
        // key zone: global index and box position
        const int lx = kl % g.T[0], ly = (kl / g.T[0]) % g.T[1], lz = kl / (g.T[0] * g.T[1]);
        const int zx = tc[0] * g.T[0] + lx, zy = tc[1] * g.T[1] + ly, zz = tc[2] * g.T[2] + lz;
        const int hx = lx + 1, hy = ly + (NB == 3 ? 1 : 0), hz = lz + (NC == 3 ? 1 : 0);
        // key-zone geometry for the zone-relative push
        const int zid[3] = {zx, zy, zz};
        double zcd[3] = {0.0, 0.0, 0.0};
        float zcf[3] = {0.f, 0.f, 0.f}, zif[3] = {0.f, 0.f, 0.f};
        float znu = 0.f, zlo = 0.f, zhi = 0.f, zhw = 0.f;
        if (kok && cnt > 0) {
#pragma unroll
            for (int d = 0; d < 3; ++d)
                if (g.n[d] > 1) {
                    zcd[d] = g.zc[d][zid[d]];
                    zcf[d] = g.zc_f[d][zid[d]];
                    zif[d] = g.ziw_f[d][zid[d]];
                }
            if (GEOM == GEOM_CYL || GEOM == GEOM_SPH) znu = g.znu_f[0][zid[0]];
            if (GEOM == GEOM_SPH) {
                zlo = g.zlo_f[1][zid[1]];
                zhi = g.zlo_f[1][zid[1] + 1];
                zhw = 0.5f / zif[1];
            }
        }
        float f[NB][NC][4], acc[NB][NC][4], S[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int b = 0; b < NB; ++b)
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                if (kok && cnt > 0)
                    smem_gas_load<float>(sgas, (hx + a - 1) + B[0] * ((hy + b - Sh::BC) + B[1] * (hz + c - Sh::CC)), f[b][c]);
                else
                    f[b][c][0] = f[b][c][1] = f[b][c][2] = f[b][c][3] = 0.f;
#pragma unroll
                for (int ch = 0; ch < 4; ++ch) acc[b][c][ch] = 0.f;
            }

        const int rounds = (maxcnt + 2) / 3;
        for (int r = 0; r < rounds; ++r) {
            const int pos = 3 * r + a;
            const bool has = kok && pos < cnt;
            const int64_t gi = off0 + pos;
            // ---- own grain: first half drift and weights, relative to the
            // key zone (fast); grains that left it take the exact path
            double q[3] = {0.0, 0.0, 0.0};
            float pn[3] = {0.f, 0.f, 0.f};
            float w[3][3] = {{0.f, 1.f, 0.f}, {0.f, 1.f, 0.f}, {0.f, 1.f, 0.f}};
            float iw[3] = {0.f, 0.f, 0.f};
            float inc1[3] = {0.f, 0.f, 0.f};
            float qf[3] = {0.f, 0.f, 0.f};  // half-step coordinates
            int host[3] = {0, 0, 0};
            int sp = 0;
            bool live = false, ingroup = false;
            if (has) {
                q[0] = A.s.q[0][gi]; q[1] = A.s.q[1][gi]; q[2] = A.s.q[2][gi];
                live = !isnan(q[0]);
                if (live) {
                    pn[0] = A.s.p[0][gi]; pn[1] = A.s.p[1][gi]; pn[2] = A.s.p[2][gi];
                    sp = A.s.species ? A.s.species[gi] : 0;
                    float u[3], zc3[3];
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        if (g.n[d] > 1) { u[d] = (float)(q[d] - zcd[d]); zc3[d] = zcf[d]; }
                        else { u[d] = 0.f; zc3[d] = (float)q[d]; }
                    }
                    // first half drift (Eq. exp_midpoint; Eq. drift1_cylindrical;
                    // spherical r, theta, phi in turn)
                    if (GEOM == GEOM_CYL) {
                        inc1[0] = h * pn[0]; u[0] += inc1[0];
                        const float R = zc3[0] + u[0];
                        inc1[1] = h * pn[1] / (R * R); u[1] += inc1[1];
                        inc1[2] = h * pn[2]; u[2] += inc1[2];
                    } else if (GEOM == GEOM_SPH) {
                        inc1[0] = h * pn[0]; u[0] += inc1[0];
                        const float r = zc3[0] + u[0];
                        inc1[1] = h * pn[1] / (r * r); u[1] += inc1[1];
                        const float st = sinf(zc3[1] + u[1]);
                        inc1[2] = h * pn[2] / (r * r * st * st); u[2] += inc1[2];
                    } else if (GEOM == GEOM_SB) {
                        inc1[0] = h * pn[0]; u[0] += inc1[0];
                        inc1[1] = A.ph.fargo ? h * (pn[1] - A.ph.q_om_f * (zc3[0] + u[0])) : h * pn[1];
                        u[1] += inc1[1];
                        inc1[2] = h * pn[2]; u[2] += inc1[2];
                    } else {
#pragma unroll
                        for (int d = 0; d < 3; ++d) { inc1[d] = h * pn[d]; u[d] += inc1[d]; }
                    }
                    float dl[3];
                    ingroup = true;
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        qf[d] = zc3[d] + u[d];
                        dl[d] = u[d] * zif[d];
                        if (g.n[d] > 1) ingroup &= fabsf(dl[d]) <= 0.50001f;
                    }
                    if (ingroup) {
                        host[0] = zx; host[1] = zy; host[2] = zz;
#pragma unroll
                        for (int d = 0; d < 3; ++d) {
                            iw[d] = zif[d];
                            if (g.n[d] <= 1) continue;
                            if ((GEOM == GEOM_CYL || GEOM == GEOM_SPH) && d == 0) {
                                if (GEOM == GEOM_CYL) w_cyl<float>(TA.tsc, dl[0], znu, w[0]);
                                else w_sphr<float>(TA.tsc, dl[0], znu, w[0]);
                            } else if (GEOM == GEOM_SPH && d == 1) {
                                w_theta<float>(TA.tsc, qf[1], zlo, zhi, u[1], zhw, w[1]);
                            } else {
                                w_cart<float>(TA.tsc, dl[d], w[d]);
                            }
                        }
                    } else {
                        // exact path: double-precision half drift, boundaries
                        // and zone search
#pragma unroll
                        for (int d = 0; d < 3; ++d) inc1[d] = 0.f;
                        drift<float, GEOM>(A.ph, q, q, pn, h, false, inc1);
                        if (!apply_bc<float, GEOM>(g, A.ph, A.ph.shift_mid, q, pn)) {
                            A.s.q[0][gi] = __longlong_as_double(0x7ff8000000000000LL);
                            ++nremoved;
                            live = false;
                        } else {
#pragma unroll
                            for (int d = 0; d < 3; ++d) {
                                zone_weights<float, GEOM>(g, d, TA.tsc, q[d], host[d], w[d], iw[d]);
                                qf[d] = (float)q[d];
                            }
                        }
                    }
                }
            }
            const bool grp_ok = live && ingroup;
            // ---- exchange weights inside the group: slot e holds the grain
            // of lane (a + e) % 3; wx is sent at the receiver's x offset
            float gx[3], gy[3][3], gz[3][3];
            bool gok[3];
            gx[0] = sel3(w[0], a);
#pragma unroll
            for (int k = 0; k < 3; ++k) { gy[0][k] = w[1][k]; gz[0][k] = w[2][k]; }
            gok[0] = grp_ok;
#pragma unroll
            for (int e = 1; e < 3; ++e) {
                const int srcl = e == 1 ? src1 : src2;
                const int want = (a + 3 - e) % 3;  // receiver's offset, seen from this lane
                gx[e] = __shfl_sync(FULL, sel3(w[0], want), srcl);
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    gy[e][k] = NB == 3 ? __shfl_sync(FULL, w[1][k], srcl) : w[1][k];
                    gz[e][k] = NC == 3 ? __shfl_sync(FULL, w[2][k], srcl) : w[2][k];
                }
                gok[e] = __shfl_sync(FULL, grp_ok ? 1 : 0, srcl) != 0;
            }
            // ---- partial gathers over this lane's slab for the three grains
            float P[3][4];
#pragma unroll
            for (int e = 0; e < 3; ++e) {
#pragma unroll
                for (int ch = 0; ch < 4; ++ch) P[e][ch] = 0.f;
#pragma unroll
                for (int b = 0; b < NB; ++b)
#pragma unroll
                    for (int c = 0; c < NC; ++c) {
                        const float wyz = gy[e][NB == 3 ? b : 1] * gz[e][NC == 3 ? c : 1];
#pragma unroll
                        for (int ch = 0; ch < 4; ++ch) P[e][ch] += wyz * f[b][c][ch];
                    }
#pragma unroll
                for (int ch = 0; ch < 4; ++ch) P[e][ch] *= gx[e];
            }
            // own grain's gather: own slab + the two other slabs
            float G[4];
#pragma unroll
            for (int ch = 0; ch < 4; ++ch) {
                const float p1 = __shfl_sync(FULL, P[2][ch], src1);
                const float p2 = __shfl_sync(FULL, P[1][ch], src2);
                G[ch] = (P[0][ch] + p1) + p2;
            }
            // ---- own grain: kick, second half drift, deposit impulse
            float D[4] = {0.f, 0.f, 0.f, 0.f};
            if (live) {
                int lb[3];
                bool inbox = true;
                if (!ingroup) {
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        int l = host[d] - o[d];
                        if (g.n[d] > 1 && g.bc[d] == DUST_BC_PERIODIC) {
                            if (l < 0) l += g.n[d];
                            else if (l >= B[d]) l -= g.n[d];
                        }
                        lb[d] = l;
                        if (g.n[d] > 1) inbox &= (l >= 1) && (l <= B[d] - 2);
                    }
                    // stale-sort grain: own 27-node gather
#pragma unroll
                    for (int ch = 0; ch < 4; ++ch) G[ch] = 0.f;
#pragma unroll
                    for (int c3 = 0; c3 < 3; ++c3) {
                        if (NC == 1 && c3 != 1) continue;
#pragma unroll
                        for (int b = 0; b < 3; ++b) {
                            if (NB == 1 && b != 1) continue;
#pragma unroll
                            for (int aa = 0; aa < 3; ++aa) {
                                const float W = w[0][aa] * (w[1][b] * w[2][c3]);
                                float fv[4];
                                if (inbox) {
                                    smem_gas_load<float>(sgas, (lb[0] + aa - 1) + B[0] * ((lb[1] + b - 1) + B[1] * (lb[2] + c3 - 1)), fv);
                                } else {
                                    const int ix = node_of(host[0], aa - 1, g.n[0], g.bc[0]);
                                    const int iy = node_of(host[1], b - 1, g.n[1], g.bc[1]);
                                    const int iz = node_of(host[2], c3 - 1, g.n[2], g.bc[2]);
                                    load_gas<float>(A.gas, ix + (int64_t)g.n[0] * (iy + (int64_t)g.n[1] * iz), fv);
                                }
#pragma unroll
                                for (int ch = 0; ch < 4; ++ch) G[ch] += W * fv[ch];
                            }
                        }
                    }
                }
                const float value = A.s.param ? A.s.param[gi] : A.sp.tau_f[sp];
                const float tau = stopping_time<float, GEOM>(A.ph, A.sp.mode[sp], value, qf, G[0]);
                const float x = dt / tau;
                const float E = expf(-x);
                const float cg = -expm1f(-x);
                const float h1 = (x == 0.f) ? dt : dt * cg / x;
                const float vg[3] = {G[1], G[2], G[3]};
                float pp[3], acc3[3], dH[3], inc2[3];
                kick<float, GEOM>(A.ph, qf, pn, vg, E, cg, h1, pp, acc3, dH);
                if (ingroup) {
                    // second half drift with the half-step metric factors, then
                    // one double-precision update by the summed increment
                    if (GEOM == GEOM_CYL) {
                        inc2[0] = h * pp[0];
                        inc2[1] = h * pp[1] / (qf[0] * qf[0]);
                        inc2[2] = h * pp[2];
                    } else if (GEOM == GEOM_SPH) {
                        const float st = sinf(qf[1]);
                        inc2[0] = h * pp[0];
                        inc2[1] = h * pp[1] / (qf[0] * qf[0]);
                        inc2[2] = h * pp[2] / (qf[0] * qf[0] * st * st);
                    } else if (GEOM == GEOM_SB) {
                        inc2[0] = h * pp[0];
                        inc2[1] = A.ph.fargo ? h * (pp[1] - A.ph.q_om_f * qf[0]) : h * pp[1];
                        inc2[2] = h * pp[2];
                    } else {
#pragma unroll
                        for (int d = 0; d < 3; ++d) inc2[d] = h * pp[d];
                    }
#pragma unroll
                    for (int d = 0; d < 3; ++d) q[d] += (double)(inc1[d] + inc2[d]);
                } else {
                    const double qm[3] = {q[0], q[1], q[2]};
                    drift<float, GEOM>(A.ph, q, qm, pp, h, true, inc2);
                }
                float pnew[3] = {pp[0], pp[1], pp[2]};
                const bool alive = apply_bc<float, GEOM>(g, A.ph, A.ph.shift_end, q, pnew);
                const float mq = A.sp.mqf[sp];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    D[c] = -mq * ((pp[c] - pn[c]) - dt * acc3[c]);
                    D[3] += D[c] * dH[c];
                }
                if (!(isfinite(pp[0]) && isfinite(pp[1]) && isfinite(pp[2])))
                    atomicOr(&A.status[ST_FLAGS], DUST_FLAG_NAN);
#pragma unroll
                for (int d = 0; d < 3; ++d) moved = fmaxf(moved, fabsf(inc1[d] + inc2[d]) * iw[d]);
                if (!ingroup) {
                    // per-grain fixed-point rule for a grain outside its key zone
                    if (inbox) {
                        long long rest[4];
#pragma unroll
                        for (int ch = 0; ch < 4; ++ch) rest[ch] = rint_to_ll(D[ch]);
                        const int hl = lb[0] + B[0] * (lb[1] + B[1] * lb[2]);
#pragma unroll
                        for (int c3 = 0; c3 < 3; ++c3) {
                            if (NC == 1 && c3 != 1) continue;
#pragma unroll
                            for (int b = 0; b < 3; ++b) {
                                if (NB == 1 && b != 1) continue;
#pragma unroll
                                for (int aa = 0; aa < 3; ++aa) {
                                    if (aa == 1 && b == 1 && c3 == 1) continue;
                                    const float W = w[0][aa] * (w[1][b] * w[2][c3]);
                                    const int lin = hl + (aa - 1) + B[0] * ((b - 1) + B[1] * (c3 - 1));
#pragma unroll
                                    for (int ch = 0; ch < 4; ++ch) {
                                        const long long piece = rint_to_ll(W * D[ch]);
                                        if (piece != 0) {
                                            atomicAdd(&sdep[ch * bvol + lin], (unsigned long long)piece);
                                            rest[ch] -= piece;
                                        }
                                    }
                                }
                            }
                        }
#pragma unroll
                        for (int ch = 0; ch < 4; ++ch)
                            if (rest[ch] != 0) atomicAdd(&sdep[ch * bvol + hl], (unsigned long long)rest[ch]);
                    } else {
                        deposit_fixed<float>(g, A.dep, host, w, D, A.status);
                    }
                }
                if (!alive) {
                    q[0] = __longlong_as_double(0x7ff8000000000000LL);
                    ++nremoved;
                }
                A.s.q[0][gi] = q[0]; A.s.q[1][gi] = q[1]; A.s.q[2][gi] = q[2];
                A.s.p[0][gi] = pnew[0]; A.s.p[1][gi] = pnew[1]; A.s.p[2][gi] = pnew[2];
            }
            // ---- deposit impulses of the group's grains into this slab
            float gD[3][4];
#pragma unroll
            for (int ch = 0; ch < 4; ++ch) {
                gD[0][ch] = D[ch];
                gD[1][ch] = __shfl_sync(FULL, D[ch], src1);
                gD[2][ch] = __shfl_sync(FULL, D[ch], src2);
            }
#pragma unroll
            for (int e = 0; e < 3; ++e) {
                if (!gok[e]) continue;
#pragma unroll
                for (int b = 0; b < NB; ++b)
#pragma unroll
                    for (int c = 0; c < NC; ++c) {
                        const float W = gx[e] * (gy[e][NB == 3 ? b : 1] * gz[e][NC == 3 ? c : 1]);
#pragma unroll
                        for (int ch = 0; ch < 4; ++ch) acc[b][c][ch] += W * gD[e][ch];
                    }
                if (a == 1) {
#pragma unroll
                    for (int ch = 0; ch < 4; ++ch) S[ch] += gD[e][ch];
                }
            }
        }

        // ---- quantise this zone's run and flush it to the deposit box
        long long ps[4] = {0, 0, 0, 0};
        if (kok && cnt > 0) {
#pragma unroll
            for (int b = 0; b < NB; ++b)
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    if (a == 1 && b == Sh::BC && c == Sh::CC) continue;  // host: remainder
                    const int lin = (hx + a - 1) + B[0] * ((hy + b - Sh::BC) + B[1] * (hz + c - Sh::CC));
#pragma unroll
                    for (int ch = 0; ch < 4; ++ch) {
                        big |= !(fabsf(acc[b][c][ch]) < 4.5e15f);
                        const long long piece = rint_to_ll(acc[b][c][ch]);
                        if (piece != 0) {
                            atomicAdd(&sdep[ch * bvol + lin], (unsigned long long)piece);
                            ps[ch] += piece;
                        }
                    }
                }
        }
#pragma unroll
        for (int ch = 0; ch < 4; ++ch) {
            const long long s1 = __shfl_sync(FULL, ps[ch], base + 0);
            const long long s2 = __shfl_sync(FULL, ps[ch], base + 2);
            if (a == 1 && kok && cnt > 0) {
                big |= !(fabsf(S[ch]) < 4.5e15f);
                const long long rest = rint_to_ll(S[ch]) - (ps[ch] + s1 + s2);
                if (rest != 0)
                    atomicAdd(&sdep[ch * bvol + hx + B[0] * (hy + B[1] * hz)], (unsigned long long)rest);
            }
        }
    }
    if (big) atomicOr(&A.status[ST_FLAGS], DUST_FLAG_OVERFLOW);
    __syncthreads();

    // ---- flush the deposit box
    for (int lin = threadIdx.x; lin < bvol; lin += blockDim.x) {
        const int bx = lin % B[0], by = (lin / B[0]) % B[1], bz = lin / (B[0] * B[1]);
        const int i = map_zone(o[0] + bx, g.n[0], g.bc[0]);
        const int j = map_zone(o[1] + by, g.n[1], g.bc[1]);
        const int k = map_zone(o[2] + bz, g.n[2], g.bc[2]);
        const int64_t gz = i + (int64_t)g.n[0] * (j + (int64_t)g.n[1] * k);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const unsigned long long v = sdep[c * bvol + lin];
            if (v != 0ull) atomicAdd(&A.dep[4 * gz + c], v);
        }
    }
    const unsigned mv = __reduce_max_sync(FULL, __float_as_uint(moved));
    const unsigned nr = __reduce_add_sync(FULL, (unsigned)nremoved);
    if (lane == 0) {
        if (mv) atomicMax(&A.status[ST_MAXMOVE], mv);
        if (nr) atomicAdd(reinterpret_cast<unsigned long long *>(&A.status[ST_REMOVED_LO]),
                          (unsigned long long)nr);
    }
}

inline size_t slab_smem_bytes(const GridDev &g)
{
    size_t bvol = 1;
    for (int d = 0; d < 3; ++d) bvol *= (size_t)(g.T[d] + (g.n[d] > 1 ? 2 : 0));
    return bvol * (4 * sizeof(float) + 4 * sizeof(long long));
}

template <int GEOM, int FLAT>
cudaError_t launch_step_slab(const TiledArgs<float> &a, cudaStream_t s)
{
    const GridDev &g = a.s.g;
    const int ntiles = g.nt[0] * g.nt[1] * g.nt[2];
    const size_t smem = slab_smem_bytes(g);
    auto kern = step_slab_kernel<GEOM, FLAT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<ntiles, kSlabThreads, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace dust
