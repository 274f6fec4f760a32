// team.cuh -- point arithmetic shared by the four warps of a 128-thread block.
//
// One warp's XYZZ addition runs its 14 F_q products one after another on the
// integer pipe of the single SM sub-partition the warp lives on, so the
// addition takes ~14 product latencies however idle the rest of the SM is.
// That sets the time of the phases where only a few additions are in flight
// (the bucket reduction's scans and trees, small bucket sets).
//
// A team spreads each point operation over the four sub-partitions: lane l
// of every warp works on the same operation l (32 operations per team), and
// the products of a formula that do not depend on one another run in
// different warps, which exchange field elements through shared memory.  An
// addition (add-2008-s) then costs 4 product latencies and a doubling
// (dbl-2008-s-1) 3, plus a block barrier per stage.
//
// Storage is a shared-memory file of F_q slots: slot s holds one element per
// lane, limb-planar (word i of lane l at f[(s * 8 + i) * 32 + l]) so that the
// 32 lanes of a warp touch 32 consecutive words.  A point takes four
// consecutive slots (X, Y, ZZ, ZZZ); infinity is ZZ = 0.
//
// Every function below is called by all 128 threads of the block with
// block-uniform arguments (it contains barriers) and ends with a barrier, so
// its result slots are visible to every warp on return.
#pragma once
#include "curve.cuh"

namespace zk {

constexpr int kTeamThreads = 128;
constexpr int kTeamTemps = 10;  // scratch slots used by team_add / team_dbl

ZK_DEV uint32_t team_lane() { return threadIdx.x & 31; }
ZK_DEV uint32_t team_warp() { return threadIdx.x >> 5; }

ZK_DEV Fq tf_load(const uint32_t *f, int s) {
    const uint32_t l = team_lane();
    Fq r;
#pragma unroll
    for (int i = 0; i < 8; i++) r.v[i] = f[(s * 8 + i) * 32 + l];
    return r;
}

ZK_DEV void tf_store(uint32_t *f, int s, const Fq &v) {
    const uint32_t l = team_lane();
#pragma unroll
    for (int i = 0; i < 8; i++) f[(s * 8 + i) * 32 + l] = v.v[i];
}

// o = 2 a (dbl-2008-s-1, a = 0) for the lanes with `mine`; other lanes keep
// o.  o may alias a.  Temps t .. t + 9.  Infinity doubles to infinity (ZZ3 =
// V ZZ = 0).
ZK_DEV void team_dbl_masked(uint32_t *f, int a, int o, int t, bool mine) {
    const uint32_t w = team_warp();
    // stage 1: V = U^2 (U = 2Y), XX = X^2
    if (w < 2) {
        Fq x = w == 0 ? fe_dbl<FqP>(tf_load(f, a + 1)) : tf_load(f, a + 0);
        tf_store(f, t + w, fe_sqr<FqP>(x));
    }
    __syncthreads();
    // stage 2: W = U V, S = X V, MM = M^2 (M = 3 XX), ZZ3 = V ZZ
    {
        Fq x, y;
        if (w == 0) {
            x = fe_dbl<FqP>(tf_load(f, a + 1));
            y = tf_load(f, t + 0);
        } else if (w == 1) {
            x = tf_load(f, a + 0);
            y = tf_load(f, t + 0);
        } else if (w == 2) {
            x = fe_mul3<FqP>(tf_load(f, t + 1));
            y = x;
        } else {
            x = tf_load(f, t + 0);
            y = tf_load(f, a + 2);
        }
        tf_store(f, t + 2 + w, fe_mul<FqP>(x, y));
    }
    __syncthreads();
    // stage 3: ZZZ3 = W ZZZ, WY = W Y, X3 = MM - 2S, MS = M (S - X3)
    if (w == 0) {
        tf_store(f, t + 6, fe_mul<FqP>(tf_load(f, t + 2), tf_load(f, a + 3)));
    } else if (w == 1) {
        tf_store(f, t + 7, fe_mul<FqP>(tf_load(f, t + 2), tf_load(f, a + 1)));
    } else if (w == 2) {
        const Fq S = tf_load(f, t + 3);
        const Fq X3 = fe_sub<FqP>(tf_load(f, t + 4), fe_dbl<FqP>(S));
        tf_store(f, t + 8, X3);
        const Fq M = fe_mul3<FqP>(tf_load(f, t + 1));
        tf_store(f, t + 9, fe_mul<FqP>(M, fe_sub<FqP>(S, X3)));
    }
    __syncthreads();
    // stage 4: warp w writes coordinate w
    if (mine) {
        Fq r;
        if (w == 0) r = tf_load(f, t + 8);
        else if (w == 1) r = fe_sub<FqP>(tf_load(f, t + 9), tf_load(f, t + 7));
        else if (w == 2) r = tf_load(f, t + 5);
        else r = tf_load(f, t + 6);
        tf_store(f, o + w, r);
    }
    __syncthreads();
}

ZK_DEV void team_dbl(uint32_t *f, int a, int o, int t) { team_dbl_masked(f, a, o, t, true); }

// o = a + b (add-2008-s) with every exceptional case: either operand
// infinite, a = b (doubling), a = -b (infinity).  o may alias a or b.  Temps
// t .. t + 9 must not overlap a, b or o.
ZK_DEV void team_add(uint32_t *f, int a, int b, int o, int t) {
    const uint32_t w = team_warp();
    // stage 1: U1 = X1 ZZ2, U2 = X2 ZZ1, S1 = Y1 ZZZ2, S2 = Y2 ZZZ1
    {
        const int p = (w & 1) ? b : a;   // point whose coordinate is taken
        const int q = (w & 1) ? a : b;   // point whose Z power multiplies it
        const int ci = (w < 2) ? 0 : 1;  // X or Y
        tf_store(f, t + w, fe_mul<FqP>(tf_load(f, p + ci), tf_load(f, q + 2 + ci)));
    }
    __syncthreads();
    // stage 2: P = U2 - U1, R = S2 - S1; PP = P^2, RR = R^2, ZZ1 ZZ2, ZZZ1 ZZZ2
    const Fq P = fe_sub<FqP>(tf_load(f, t + 1), tf_load(f, t + 0));
    const Fq R = fe_sub<FqP>(tf_load(f, t + 3), tf_load(f, t + 2));
    const bool inf_a = fe_is_zero<FqP>(tf_load(f, a + 2));
    const bool inf_b = fe_is_zero<FqP>(tf_load(f, b + 2));
    const bool pz = fe_is_zero<FqP>(P);
    const bool rz = fe_is_zero<FqP>(R);
    {
        Fq x, y;
        if (w == 0) {
            x = P;
            y = P;
        } else if (w == 1) {
            x = R;
            y = R;
        } else {
            x = tf_load(f, a + w);  // ZZ1 (w = 2) or ZZZ1 (w = 3)
            y = tf_load(f, b + w);
        }
        tf_store(f, t + 4 + w, fe_mul<FqP>(x, y));
    }
    __syncthreads();
    // stage 3: PPP = P PP, Q = U1 PP, ZZ3 = ZZ1 ZZ2 PP
    if (w < 3) {
        const Fq PP = tf_load(f, t + 4);
        const Fq y = w == 0 ? P : (w == 1 ? tf_load(f, t + 0) : tf_load(f, t + 6));
        tf_store(f, w == 0 ? t + 8 : (w == 1 ? t + 9 : t + 6), fe_mul<FqP>(PP, y));
    }
    __syncthreads();
    // stage 4: ZZZ3 = ZZZ1 ZZZ2 PPP, T = S1 PPP, X3 = RR - PPP - 2Q,
    // V = R (Q - X3)
    if (w == 0) {
        tf_store(f, t + 7, fe_mul<FqP>(tf_load(f, t + 7), tf_load(f, t + 8)));
    } else if (w == 1) {
        tf_store(f, t + 0, fe_mul<FqP>(tf_load(f, t + 2), tf_load(f, t + 8)));
    } else if (w == 2) {
        const Fq Q = tf_load(f, t + 9);
        const Fq X3 = fe_sub<FqP>(fe_sub<FqP>(tf_load(f, t + 5), tf_load(f, t + 8)), fe_dbl<FqP>(Q));
        tf_store(f, t + 5, X3);
        tf_store(f, t + 4, fe_mul<FqP>(R, fe_sub<FqP>(Q, X3)));
    }
    __syncthreads();
    // stage 5: warp w writes coordinate w of the result.
    const bool need_dbl = !inf_a && !inf_b && pz && rz;
    if (!need_dbl) {
        Fq r;
        if (inf_a) {
            r = tf_load(f, b + w);
        } else if (inf_b) {
            r = tf_load(f, a + w);
        } else if (pz) {
            r = fe_zero<FqP>();  // a = -b
        } else if (w == 0) {
            r = tf_load(f, t + 5);
        } else if (w == 1) {
            r = fe_sub<FqP>(tf_load(f, t + 4), tf_load(f, t + 0));
        } else {
            r = tf_load(f, t + 4 + w);  // ZZ3 (t + 6) or ZZZ3 (t + 7)
        }
        tf_store(f, o + w, r);
    }
    // The lanes with a = b left o untouched (and so a, when o aliases it).
    if (__syncthreads_or(need_dbl)) team_dbl_masked(f, a, o, t, need_dbl);
}

// dst = src shifted down by d lanes: lane l receives lane l + d, lanes with
// l + d >= 32 receive infinity.  dst must differ from src.
ZK_DEV void team_shift(uint32_t *f, int src, int dst, int d) {
    const uint32_t w = team_warp(), l = team_lane();
    uint32_t v[8];
#pragma unroll
    for (int i = 0; i < 8; i++) v[i] = (l + d < 32) ? f[((src + w) * 8 + i) * 32 + l + d] : 0u;
#pragma unroll
    for (int i = 0; i < 8; i++) f[((dst + w) * 8 + i) * 32 + l] = v[i];
    __syncthreads();
}

// dst = keep ? src : infinity, lane by lane.
ZK_DEV void team_copy(uint32_t *f, int src, int dst, bool keep) {
    const uint32_t w = team_warp();
    tf_store(f, dst + w, keep ? tf_load(f, src + w) : fe_zero<FqP>());
    __syncthreads();
}

// Point slots p = infinity (no barrier: callers batch these before one).
ZK_DEV void team_set_inf_nosync(uint32_t *f, int p) { tf_store(f, p + team_warp(), fe_zero<FqP>()); }

// Coordinate `team_warp()` of the XYZZ point at src (Montgomery form, 128
// bytes), or zero when !valid: what this warp stores for its lane.
ZK_DEV Fq team_fetch(const Xyzz *src, bool valid) {
    if (!valid) return fe_zero<FqP>();
    return fe_load<FqP>(reinterpret_cast<const char *>(src) + 32 * team_warp());
}

// Writes coordinate `team_warp()` of the point in slots p to dst.
ZK_DEV void team_put(const uint32_t *f, int p, Xyzz *dst) {
    fe_store<FqP>(reinterpret_cast<char *>(dst) + 32 * team_warp(), tf_load(f, p + team_warp()));
}

// The point in slots p of lane `lane` (any thread may call it after a
// barrier).
ZK_DEV Xyzz team_point_of(const uint32_t *f, int p, uint32_t lane) {
    Xyzz r;
#pragma unroll
    for (int i = 0; i < 8; i++) {
        r.X.v[i] = f[((p + 0) * 8 + i) * 32 + lane];
        r.Y.v[i] = f[((p + 1) * 8 + i) * 32 + lane];
        r.ZZ.v[i] = f[((p + 2) * 8 + i) * 32 + lane];
        r.ZZZ.v[i] = f[((p + 3) * 8 + i) * 32 + lane];
    }
    return r;
}

// The point in slots p for the calling thread's lane, gathered from the
// four coordinates (any warp may call it after a barrier).
ZK_DEV Xyzz team_point(const uint32_t *f, int p) {
    Xyzz r;
    r.X = tf_load(f, p + 0);
    r.Y = tf_load(f, p + 1);
    r.ZZ = tf_load(f, p + 2);
    r.ZZZ = tf_load(f, p + 3);
    return r;
}

}  // namespace zk
