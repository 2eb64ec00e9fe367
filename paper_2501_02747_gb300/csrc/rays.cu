// rays.cu -- validation of image-tree candidates as specular rays, by the
// image method (Sec. IV-B: the candidates of the pre-processed image tree and
// the brute-force method give the same valid rays).  Faces must be
// axis-aligned rectangles (the caller checks).
//
// Candidate (t, k, f1..fk), source T = Tx_t and receiver R = Rx_t, scaled by
// 2s.  Face f_m is the plane x_a = c (a, c integers) with the rectangle
// [lo, hi] on the other two axes; its mirror maps x_a to 2c - x_a, so every
// image is an integer point: I_0 = T, I_m = mirror_m(I_(m-1)).  The unfolded
// ray is the segment from R (parameter 0) to I_k (parameter 1).  Leg m of the
// ray, from P_m to P_(m+1) (P_0 = T, P_(k+1) = R), is that segment carried
// back through mirrors m+1..k: the integer line U_m + mu V_m with U_k = R,
// U_(m-1) = mirror_m(U_m) and V_m = I_m - U_m, over mu in (mu_(m+1), mu_m),
// where mu_m is where U_m + mu V_m meets the plane of f_m, mu_(k+1) = 0 and
// mu_0 = 1.  The candidate is a ray when
//   0 < mu_k < ... < mu_1 < 1            (each P_m strictly between P_(m+1) and I_m),
//   P_m lies in the closed face f_m,
//   I_(m-1) and P_(m+1) are strictly in front of f_m (outward incidence),
//   no face meets any open leg.
// Coordinates stay below 2^26 and parameters are fractions of integers below
// 2^27, so every test compares 64-bit products exactly.
#include "rays.cuh"
#include "traverse.cuh"

namespace ivm {

namespace {

struct Frac {
    long long n, d;   // d > 0
};

__device__ __forceinline__ bool lt(Frac x, Frac y) { return x.n * y.d < y.n * x.d; }

__device__ __forceinline__ Frac frac(long long n, long long d)
{
    return d < 0 ? Frac{-n, -d} : Frac{n, d};
}

// Axis-aligned face of a leaf: plane axis, its offset, in-plane bounds.
struct Rect {
    int a, b0, b1;
    int c, lo0, hi0, lo1, hi1;
    int sig;   // +1: the outward normal points along +a
};

__device__ __forceinline__ int pick(int x, int y, int z, int i) { return i == 0 ? x : (i == 1 ? y : z); }

__device__ __forceinline__ Rect rect_of(const Leaf &L)
{
    Rect r;
    r.a = L.nx != 0 ? 0 : (L.ny != 0 ? 1 : 2);
    r.sig = pick(L.nx, L.ny, L.nz, r.a) > 0 ? 1 : -1;
    r.b0 = r.a == 0 ? 1 : 0;
    r.b1 = r.a == 2 ? 1 : 2;
    r.c = pick(L.ox, L.oy, L.oz, r.a);
    const int o0 = pick(L.ox, L.oy, L.oz, r.b0), o1 = pick(L.ox, L.oy, L.oz, r.b1);
    const int e0 = pick(L.ux, L.uy, L.uz, r.b0) + pick(L.vx, L.vy, L.vz, r.b0);
    const int e1 = pick(L.ux, L.uy, L.uz, r.b1) + pick(L.vx, L.vy, L.vz, r.b1);
    r.lo0 = min(o0, o0 + e0); r.hi0 = max(o0, o0 + e0);
    r.lo1 = min(o1, o1 + e1); r.hi1 = max(o1, o1 + e1);
    return r;
}

struct I3 {
    long long v[3];
};

// Does face F meet the open part mu in (lo, hi) of the line U + mu V?
__device__ bool leg_meets(const I3 &U, const I3 &V, Frac lo, Frac hi, const Rect &F)
{
    const long long Ua = U.v[F.a], Va = V.v[F.a];
    const long long U0 = U.v[F.b0], V0 = V.v[F.b0], U1 = U.v[F.b1], V1 = V.v[F.b1];
    if (Va != 0) {   // crosses the plane once
        const Frac m = frac(F.c - Ua, Va);
        if (!(lt(lo, m) && lt(m, hi))) return false;
        const long long x0 = U0 * m.d + m.n * V0, x1 = U1 * m.d + m.n * V1;
        return (long long)F.lo0 * m.d <= x0 && x0 <= (long long)F.hi0 * m.d &&
               (long long)F.lo1 * m.d <= x1 && x1 <= (long long)F.hi1 * m.d;
    }
    if (Ua != F.c) return false;
    // the line lies in the face's plane: parameters inside the closed rectangle
    bool has_lo = false, has_hi = false;
    Frac plo = {0, 1}, phi = {0, 1};
    const long long Us[2] = {U0, U1}, Vs[2] = {V0, V1};
    const int los[2] = {F.lo0, F.lo1}, his[2] = {F.hi0, F.hi1};
    for (int i = 0; i < 2; i++) {
        if (Vs[i] == 0) {
            if (Us[i] < los[i] || Us[i] > his[i]) return false;
            continue;
        }
        Frac e = frac(los[i] - Us[i], Vs[i]), f = frac(his[i] - Us[i], Vs[i]);
        if (lt(f, e)) { Frac t = e; e = f; f = t; }
        if (!has_lo || lt(plo, e)) { plo = e; has_lo = true; }
        if (!has_hi || lt(f, phi)) { phi = f; has_hi = true; }
    }
    if (has_lo && has_hi && lt(phi, plo)) return false;
    return (!has_lo || lt(plo, hi)) && (!has_hi || lt(lo, phi));
}

// Leg walks use the integer segment U_m -> U_m + V_m, whose coordinates can
// exceed 2^24 (images lie outside the scene) and so round in float: every
// box is widened by 64 units (directed rounding) to keep the test a superset.
struct WideBoxes {
    __device__ __forceinline__ bool node(int) const { return true; }
    __device__ __forceinline__ void grow(float &ax, float &ay, float &az, float &bx, float &by,
                                         float &bz) const
    {
        ax = __fsub_rd(ax, 64.f); ay = __fsub_rd(ay, 64.f); az = __fsub_rd(az, 64.f);
        bx = __fadd_ru(bx, 64.f); by = __fadd_ru(by, 64.f); bz = __fadd_ru(bz, 64.f);
    }
};

// Leaf test of a leg walk: true when the face meets the lane's leg.
struct LegLeaf {
    const I3 *U, *V;
    const Frac *lo, *hi;
    __device__ __forceinline__ bool operator()(const Seg &, const Leaf &L, WalkCounters &wc) const
    {
        wc.exact++;
        return leg_meets(*U, *V, *lo, *hi, rect_of(L));
    }
};

__device__ __forceinline__ void mirror(I3 &X, const Rect &F) { X.v[F.a] = 2LL * F.c - X.v[F.a]; }

}  // namespace

__global__ void k_validate(DevScenes g, RayArgs a, int *err)
{
    const int lane = threadIdx.x & 31;
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p - lane >= a.n_paths) return;   // uniform per warp
    const SceneDesc &D = g.desc[0];
    const int K = a.max_order;
    bool ok = p < a.n_paths;
    int k = 0;
    I3 U[kRayMaxOrder + 1], V[kRayMaxOrder + 1];
    Frac mu[kRayMaxOrder + 2];
    if (ok) {
        const int *rec = a.paths + p * (K + 2);
        const long long t = rec[0];
        k = rec[1];
        if (t < 0 || t >= a.n_snap || k < 0 || k > K) {
            raise_error(err, IVM_ERR_ARG);
            ok = false;
        }
        Rect F[kRayMaxOrder + 1];
        I3 I[kRayMaxOrder + 1];
        for (int m = 1; ok && m <= k; m++) {
            const int f = rec[1 + m];
            if (f < 0 || f >= D.n) {
                raise_error(err, IVM_ERR_ARG);
                ok = false;
                break;
            }
            F[m] = rect_of(load_leaf(g.leaf, D.facet0 + f));
        }
        const long long s2 = 2LL * D.s;
        I3 T, R;
        for (int i = 0; ok && i < 3; i++) {
            T.v[i] = s2 * a.tx[3 * t + i];
            R.v[i] = s2 * a.rx[3 * t + i];
            if (T.v[i] <= -kCoordLimit || T.v[i] >= kCoordLimit || R.v[i] <= -kCoordLimit ||
                R.v[i] >= kCoordLimit) {
                raise_error(err, IVM_ERR_RANGE);
                ok = false;
            }
        }
        if (ok) {
            I[0] = T;
            for (int m = 1; m <= k; m++) {
                I[m] = I[m - 1];
                mirror(I[m], F[m]);
            }
            U[k] = R;
            for (int m = k; m >= 1; m--) {
                U[m - 1] = U[m];
                mirror(U[m - 1], F[m]);
            }
            for (int m = 0; m <= k; m++)
                for (int i = 0; i < 3; i++) V[m].v[i] = I[m].v[i] - U[m].v[i];
            mu[k + 1] = Frac{0, 1};
            mu[0] = Frac{1, 1};
            for (int m = k; ok && m >= 1; m--) {
                const Rect &Fm = F[m];
                const long long Va = V[m].v[Fm.a];
                if (Va == 0) { ok = false; break; }
                mu[m] = frac(Fm.c - U[m].v[Fm.a], Va);
                // strictly after the previous point along the unfolded ray
                if (!lt(mu[m + 1], mu[m])) { ok = false; break; }
                // P_m in the closed face
                const long long x0 = U[m].v[Fm.b0] * mu[m].d + mu[m].n * V[m].v[Fm.b0];
                const long long x1 = U[m].v[Fm.b1] * mu[m].d + mu[m].n * V[m].v[Fm.b1];
                if (x0 < (long long)Fm.lo0 * mu[m].d || x0 > (long long)Fm.hi0 * mu[m].d ||
                    x1 < (long long)Fm.lo1 * mu[m].d || x1 > (long long)Fm.hi1 * mu[m].d) {
                    ok = false;
                    break;
                }
                // outward incidence: the image I_(m-1) and the point P_(m+1) in front
                const long long si = Fm.sig * (I[m - 1].v[Fm.a] - Fm.c);
                const long long sp = Fm.sig * (U[m].v[Fm.a] * mu[m + 1].d +
                                               mu[m + 1].n * V[m].v[Fm.a] -
                                               (long long)Fm.c * mu[m + 1].d);
                if (si <= 0 || sp <= 0) { ok = false; break; }
            }
            if (ok && !lt(mu[1], mu[0])) ok = false;
        }
    }
    // legs, one walk per leg index for the warp's candidates that still hold
    for (int j = 0; j <= K; j++) {
        const bool mine = ok && j <= k;
        const unsigned alive = __ballot_sync(kFull, mine);
        if (!alive) continue;
        int px = 0, py = 0, pz = 0, qx = 0, qy = 0, qz = 0;
        if (mine) {
            px = (int)U[j].v[0]; py = (int)U[j].v[1]; pz = (int)U[j].v[2];
            qx = (int)(U[j].v[0] + V[j].v[0]);
            qy = (int)(U[j].v[1] + V[j].v[1]);
            qz = (int)(U[j].v[2] + V[j].v[2]);
        }
        Seg sg = make_seg(px, py, pz, qx, qy, qz);
        finish_seg(sg);
        const int lead = __ffs(alive) - 1;
        const float dx = (float)__shfl_sync(kFull, sg.dx, lead);
        const float dy = (float)__shfl_sync(kFull, sg.dy, lead);
        const float dz = (float)__shfl_sync(kFull, sg.dz, lead);
        WalkCounters wc;
        int blocker, myblk = -1;
        const int jj = mine ? j : 0;
        const unsigned free_lanes =
            walk_packet(sg, alive, g.nodes, g.leaf, D.root, dx, dy, dz, D.budget, err, wc,
                        LegLeaf{&U[jj], &V[jj], &mu[jj + 1], &mu[jj]}, blocker, myblk,
                        WideBoxes{});
        if (mine && !((free_lanes >> lane) & 1u)) ok = false;
    }
    if (p < a.n_paths) a.valid[p] = ok ? 1 : 0;
}

cudaError_t rays_validate(const DevScenes &g, const RayArgs &a, int *err, cudaStream_t st)
{
    if (a.n_paths == 0) return cudaSuccess;
    k_validate<<<(unsigned)((a.n_paths + 127) / 128), 128, 0, st>>>(g, a, err);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace ivm
