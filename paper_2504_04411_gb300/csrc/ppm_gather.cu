// ppm_gather.cu -- per-hit-point gather, ANOVA F-test and update (Sec. 5.1
// steps 2-4), hit points in spatial (3D Hilbert) order, blocks of 64
// threads, one hit point a thread in the epilogue.
//
// Per hit point h with radius r (this iteration's r_i):
//   * candidates: the photons of the grid cells overlapping the sphere's
//     bounding box, each row of cells trimmed to the chord of the sphere at
//     the row's nearest point; per candidate: closed-disk test d2 <= r^2 with
//     dx = x_h - x_p, then the same-surface test (snorm8 normal dot > 8064),
//     then the map of Eq. (map-function) y = (<x_h - x_p, u>, <x_h - x_p, v>),
//     the equi-areal annulus (2 |y|^2 < r^2 -> inner) and the 60-degree
//     sector by exact sign logic against sqrt(3); group = annulus * 6 +
//     sector.  These decisions use one fixed FP32 operation sequence
//     (explicit fma / _rn intrinsics, no contraction): reproducible bit for
//     bit on any device and by the CPU oracle;
//   * per group: count and (sum psi, sum psi^2) in shared memory, laid
//     out [slot][thread] so a warp's accesses hit distinct banks; the
//     iteration's flux Phi_i and pair count are the sums over groups
//     (no per-pair flux accumulator unless RGB flux is tested on luminance);
//   * epilogue: window sums += this iteration's sums, F of Eq.
//     (f-statistic) with m = t' J samples per group, compared with F_c(t')
//     (FP64 table); tau += Phi_i / (pi r_i^2) in FP64; on rejection Eq.
//     (radiusupdate) and the window is cleared (Sec. 5.1);
//   * VCM+: every pair's psi and flux carry the balance-heuristic merge
//     weight w = 1 / (1 + R_VM + R_VC / (n_VM pi r^2)) of Eq. (mis-weight).
//
// Traversals (ppm_params.mapping):
//   0  thread-owned: each thread walks the cells of its own sphere;
//   1, 2  warp-union (queues of 32 / 64 entries per lane): the warp walks
//      the union of its 32 spheres' cells
//      (skipping rows no lane needs), loads 32 photons at a time into shared
//      memory with one coalesced load and every lane tests each one
//      (broadcast reads, no divergence in the test loop); in-disk hits are
//      queued per lane and processed in lockstep when a queue fills, so the
//      long in-disk path runs with most lanes active.  Warps whose union is
//      wider than a hash block fall back to traversal 0;
//   3  warp-union with a warp-level pair queue: as 1 above, but in-disk
//      pairs go to one queue per warp (ballot + prefix) and are classified
//      32 at a time by any lane, accumulating into the owner's group sums
//      as 64-bit fixed point with shared-memory atomics (exact and
//      order-independent, hence deterministic); one tested channel;
//   4  warp per hit point: the warp takes its 32 hit points in turn, the
//      lanes split each trimmed row segment's photons into per-lane partial
//      sums, and a shuffle reduce-scatter gathers the 36 group sums into
//      the hit point's slots; one flux channel (otherwise it runs as 0).
// A context that writes the proposer's features always runs traversal 0,
// compiled separately so the other kernels carry none of that code; so does
// a context whose radii follow CPPM's chi-square test of the counts
// (ppm_params.test = 1) instead of the F-test.
#include "ppm_gather_impl.cuh"

namespace {

__global__ void k_radiance(int64_t nh, int nch, const double* __restrict__ tau,
                           const uint32_t* __restrict__ orig, double inv_iter,
                           float* __restrict__ out)
{
    const int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= nh) return;
    const int64_t o = orig[h];
    for (int c = 0; c < nch; ++c) out[o * nch + c] = (float)(tau[h * nch + c] * inv_iter);
}

template <int NCH, int NTC, bool NORMALS, bool VCM>
void launch_warp_per_hit(ppm_ctx* c, const GatherArgs& a, const Prob& pr, unsigned nb)
{
    if constexpr (NCH == 1) k_gather_update<1, NTC, NORMALS, VCM, 4><<<nb, kThreads, 0, c->stream>>>(a, pr);
}

template <int NCH, int NTC, bool NORMALS, bool VCM>
int launch_gather(ppm_ctx* c, const GatherArgs& a, const Prob& pr)
{
    const unsigned nb = (unsigned)((c->nh + kThreads - 1) / kThreads);
    const int m = c->prm.mapping;
    if (c->prm.test) {   // CPPM's count test: traversal 0, one tested channel
        if constexpr (NTC == 1)
            k_gather_update<NCH, 1, NORMALS, VCM, 0, false, true><<<nb, kThreads, 0, c->stream>>>(a, pr);
    } else if (a.feat)   // features: traversal 0 (results do not depend on the traversal)
        k_gather_update<NCH, NTC, NORMALS, VCM, 0, true><<<nb, kThreads, 0, c->stream>>>(a, pr);
    else if (m == 1)
        k_gather_update<NCH, NTC, NORMALS, VCM, 1><<<nb, kThreads, 0, c->stream>>>(a, pr);
    else if (m == 2)
        k_gather_update<NCH, NTC, NORMALS, VCM, 2><<<nb, kThreads, 0, c->stream>>>(a, pr);
    else if (m == 3 && NTC == 1)   // traversal 3 tests one channel
        k_gather_update<NCH, 1, NORMALS, VCM, 3><<<nb, kThreads, 0, c->stream>>>(a, pr);
    else if (m == 4 && NCH == 1)   // traversal 4 gathers one flux channel
        launch_warp_per_hit<NCH, NTC, NORMALS, VCM>(c, a, pr, nb);
    else
        k_gather_update<NCH, NTC, NORMALS, VCM, 0><<<nb, kThreads, 0, c->stream>>>(a, pr);
    PPM_LAUNCH_CHECK();
    return PPM_OK;
}

}  // namespace

int ppm_gather_launch(ppm_ctx* c, float bound)
{
    if (c->nh == 0) return PPM_OK;
    GatherArgs a;
    a.nh = c->nh;
    a.hp_pos = c->hp_pos; a.hp_u = c->hp_u; a.hp_v = c->hp_v;
    a.r = c->r; a.t = c->t; a.F = c->F; a.tau = c->tau;
    a.cnt = c->cnt; a.S = c->S; a.Q = c->Q;
    a.cell_start = c->cell_start;
    // with both rec1 and aux records the grid keeps them side by side in rec1
    a.rec0 = c->rec0; a.rec1 = c->rec1;
    a.aux = ((c->nch == 3 || c->prm.vcm) && c->ph_aux) ? reinterpret_cast<const uint4*>(c->rec1 + 1) : c->aux;
    a.err = c->err_dev;
    a.feat = c->feat;
    Prob pr;
    pr.geom = c->geom_dev;
    pr.fc = c->fc;
    pr.fm = c->fm;
    pr.rmax_next = c->rmax + (c->rmax_cur ^ 1);
    pr.counters = c->counters;
    pr.k = c->prm.k;
    pr.bound = bound;
    pr.n_vm = c->prm.n_vm > 0.f ? c->prm.n_vm : (float)c->J;
    pr.fc_max = c->fc_upto;
    pr.pid = 0u;
    pr.inv_r0 = 1.0f / c->r0;
    pr.log_iter = logf((float)(c->iter + 1));
    const bool nrm = c->use_normals;
    const bool vcm = c->prm.vcm != 0;
    if (c->nch == 1) {
        if (vcm) return nrm ? launch_gather<1, 1, true, true>(c, a, pr) : launch_gather<1, 1, false, true>(c, a, pr);
        return nrm ? launch_gather<1, 1, true, false>(c, a, pr) : launch_gather<1, 1, false, false>(c, a, pr);
    }
    if (c->ntc == 3) {
        if (vcm) return nrm ? launch_gather<3, 3, true, true>(c, a, pr) : launch_gather<3, 3, false, true>(c, a, pr);
        return nrm ? launch_gather<3, 3, true, false>(c, a, pr) : launch_gather<3, 3, false, false>(c, a, pr);
    }
    if (vcm) return nrm ? launch_gather<3, 1, true, true>(c, a, pr) : launch_gather<3, 1, false, true>(c, a, pr);
    return nrm ? launch_gather<3, 1, true, false>(c, a, pr) : launch_gather<3, 1, false, false>(c, a, pr);
}

int ppm_radiance_launch(ppm_ctx* c, float* out)
{
    if (c->nh == 0) return PPM_OK;
    const double inv = c->iter > 0 ? 1.0 / c->iter : 0.0;
    k_radiance<<<(unsigned)((c->nh + 255) / 256), 256, 0, c->stream>>>(c->nh, c->nch, c->tau, c->hp_orig, inv, out);
    PPM_LAUNCH_CHECK();
    return PPM_OK;
}
