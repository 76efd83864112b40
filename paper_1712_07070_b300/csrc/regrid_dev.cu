// regrid_dev.cu -- the AMR bookkeeping of GAMER-2 section 2.1 on the device:
// regridding one level (child selection from the refinement flags with proper
// nesting and the keep-for-nesting rule, canonical group numbering, the new
// level's corner / parent / sibling / child tables, its data from the old
// children or by interpolation from the parent), the neighbour (gather) plan
// of a level with its coarse-fine ghost patches (section 3.2), and the
// coarse-fine flux register maps, fix-up and restriction lists of the
// section 2.2 synchronisation.
//
// Everything is integer work over dense per-level patch-position maps and
// prefix sums, so a regrid leaves the host only the counts it needs to size
// buffers: one small device-to-host read when the refined set is unchanged,
// two when it changed.  Group numbering, ghost-patch numbering and register
// numbering are deterministic (dense position order), so every run builds
// the same hierarchy, and the numbering never changes a computed value.
#include <cuda_runtime.h>

#include <algorithm>

#include <cstring>

#include "amr_hydro.h"
#include "ctx.h"
#include "step_kernel.cuh"

namespace amrh {
namespace {

constexpr int SCAN_NT = 1024, SCAN_PER = 4, SCAN_BLOCK = SCAN_NT * SCAN_PER;

__device__ __forceinline__ int wrapd(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }
__device__ __forceinline__ int sib_kd(int dx, int dy, int dz) {
    const int k = (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1);
    return k - (k > 13);
}
__device__ __forceinline__ int face_sib_d(int f) {
    int d[3] = {0, 0, 0};
    d[f >> 1] = (f & 1) ? 1 : -1;
    return sib_kd(d[0], d[1], d[2]);
}
__device__ __forceinline__ int64_t pos_index(int px, int py, int pz, int PX, int PY) {
    return ((int64_t)pz * PY + py) * PX + px;
}

// ---- exclusive prefix sums of int32 counts (flags 1: nonzero counts as one; 2: zero
// counts as one, nonzero as none) ----

// One block per SCAN_BLOCK values; its total into bsum (one block: into
// *total, and the scan is complete).
__global__ void __launch_bounds__(SCAN_NT) k_scan_block(const int32_t *__restrict__ in, int32_t *__restrict__ out,
                                                        int32_t *__restrict__ bsum, int n, int flags,
                                                        int32_t *__restrict__ total) {
    __shared__ int32_t ws[SCAN_NT / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t base = (int64_t)blockIdx.x * SCAN_BLOCK + (int64_t)tid * SCAN_PER;
    int32_t v[SCAN_PER], s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_PER; k++) {
        const int64_t i = base + k;
        int32_t x = i < n ? in[i] : 0;
        if (flags == 1) x = x != 0;
        else if (flags == 2) x = i < n && x == 0;
        v[k] = s;
        s += x;
    }
    int32_t incl = s;  // inclusive scan of the thread totals over the warp
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) ws[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int32_t w = lane < SCAN_NT / 32 ? ws[lane] : 0, wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < SCAN_NT / 32) ws[lane] = wi - w;  // exclusive warp offsets
        if (lane == SCAN_NT / 32 - 1) {
            if (gridDim.x == 1) *total = wi;
            else bsum[blockIdx.x] = wi;
        }
    }
    __syncthreads();
    const int32_t off = ws[warp] + incl - s;
#pragma unroll
    for (int k = 0; k < SCAN_PER; k++) {
        const int64_t i = base + k;
        if (i < n) out[i] = off + v[k];
    }
}

// exclusive scan of the nb block sums in place (one block); total -> *total
__global__ void k_scan_sums(int32_t *bsum, int nb, int32_t *total) {
    __shared__ int32_t carry;
    __shared__ int32_t ws[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) carry = 0;
    __syncthreads();
    for (int c0 = 0; c0 < nb; c0 += SCAN_NT) {
        const int i = c0 + tid;
        const int32_t x = i < nb ? bsum[i] : 0;
        int32_t incl = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) ws[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            const int32_t w = ws[lane];
            int32_t wi = w;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int32_t y = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o) wi += y;
            }
            ws[lane] = wi - w;
        }
        __syncthreads();
        const int32_t ex = carry + ws[warp] + incl - x;
        __syncthreads();
        if (i < nb) bsum[i] = ex;
        if (tid == SCAN_NT - 1) carry = ex + x;
        __syncthreads();
    }
    if (tid == 0) *total = carry;
}

__global__ void k_scan_add(int32_t *__restrict__ out, const int32_t *__restrict__ bsum, int n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += bsum[i / SCAN_BLOCK];
}

// ---- patch-position maps ---------------------------------------------------------------

__global__ void k_posmap_scatter(int32_t *__restrict__ posmap, const int32_t *__restrict__ corner, int n, int PX,
                                 int PY) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x)
        posmap[pos_index(corner[3 * s] >> 3, corner[3 * s + 1] >> 3, corner[3 * s + 2] >> 3, PX, PY)] = s;
}

// ---- regrid of level l: children of level l -> level l+1 ----------------------------

// keep[q] = 1 for every level-l patch q holding a 26-neighbour position of a
// refined level-(l+1) patch (which must therefore stay refined)
__global__ void k_rg_keep(const int32_t *__restrict__ fcorner, const int32_t *__restrict__ fchild, int nf,
                          const int32_t *__restrict__ posmap_l, int PX, int PY, int PZ, int32_t *__restrict__ keep,
                          int32_t *err) {
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < nf; x += gridDim.x * blockDim.x) {
        if (fchild[x] < 0) continue;
        const int X = fcorner[3 * x] >> 3, Y = fcorner[3 * x + 1] >> 3, Z = fcorner[3 * x + 2] >> 3;
        for (int dz = -1; dz <= 1; dz++)
            for (int dy = -1; dy <= 1; dy++)
                for (int dx = -1; dx <= 1; dx++) {
                    const int qx = wrapd(X + dx, 2 * PX) >> 1, qy = wrapd(Y + dy, 2 * PY) >> 1,
                              qz = wrapd(Z + dz, 2 * PZ) >> 1;
                    const int32_t q = posmap_l[pos_index(qx, qy, qz, PX, PY)];
                    if (q < 0) atomicOr(err, 1);
                    else keep[q] = 1;
                }
    }
}

// chosen parents: flagged with all 26 siblings present, or kept with children
__global__ void k_rg_select(const uint8_t *__restrict__ pflag, const int32_t *__restrict__ sib,
                            const int32_t *__restrict__ child, const int32_t *__restrict__ keep,
                            const int32_t *__restrict__ corner, int n, int PX, int PY, int32_t *__restrict__ mark) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        bool nest_ok = true;
        for (int k = 0; k < 26; k++) nest_ok = nest_ok && sib[(int64_t)s * 26 + k] >= 0;
        const bool chosen = (pflag[s] && nest_ok) || (keep && keep[s] && child[s] >= 0);
        if (chosen) mark[pos_index(corner[3 * s] >> 3, corner[3 * s + 1] >> 3, corner[3 * s + 2] >> 3, PX, PY)] = 1;
    }
}

// Whether the set of chosen parents differs from the current children's
// parents (changed), and how many there are (count).
__global__ void k_rg_classify(const int32_t *__restrict__ mark, const int32_t *__restrict__ corner,
                              const int32_t *__restrict__ child, int n, int PX, int PY, int32_t *changed,
                              int32_t *count) {
    int cnt = 0, chg = 0;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        const int chosen = mark[pos_index(corner[3 * s] >> 3, corner[3 * s + 1] >> 3, corner[3 * s + 2] >> 3, PX, PY)];
        cnt += chosen;
        chg |= chosen != (child[s] >= 0);
    }
    if (cnt) atomicAdd(count, cnt);
    if (chg) atomicOr(changed, 1);
}

// Group numbers of the new level (ng groups), keeping slots in place: an
// existing child group keeps its number when it is below ng (taken); the
// others (moved: numbers >= ng, by number; new: parents without children, in
// (z, y, x) position order through nflag) take the free numbers below ng in
// increasing order, the moved ones first.  Pass 1 marks; pass 2 assigns.
__global__ void k_rg_keepmark(const int32_t *__restrict__ mark, const int32_t *__restrict__ corner,
                              const int32_t *__restrict__ child, int n, int PX, int PY, int ng,
                              int32_t *__restrict__ gnew, int32_t *__restrict__ gpar, int32_t *__restrict__ taken,
                              int32_t *__restrict__ mflag, int32_t *__restrict__ nflag) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        const int64_t p = pos_index(corner[3 * s] >> 3, corner[3 * s + 1] >> 3, corner[3 * s + 2] >> 3, PX, PY);
        const int og = child[s];
        gnew[s] = -1;
        if (!mark[p]) continue;
        if (og >= 0 && og < ng) {  // stays
            taken[og] = 1;
            gnew[s] = og;
            gpar[og] = s;
        } else if (og >= 0) {
            mflag[og] = 1;
        } else {
            nflag[p] = 1;
        }
    }
}

// work[rank of the parent's position among the chosen] = group: the new
// level's groups in (z, y, x) position order.
__global__ void k_rg_order(const int32_t *__restrict__ mark, const int32_t *__restrict__ prank,
                           const int32_t *__restrict__ corner, const int32_t *__restrict__ gnew, int n, int PX, int PY,
                           int32_t *__restrict__ work) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        const int64_t p = pos_index(corner[3 * s] >> 3, corner[3 * s + 1] >> 3, corner[3 * s + 2] >> 3, PX, PY);
        if (mark[p]) work[prank[p]] = gnew[s];
    }
}

__global__ void k_rg_freelist(int ng, const int32_t *__restrict__ taken, const int32_t *__restrict__ frank,
                              int32_t *__restrict__ flist) {
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < ng; g += gridDim.x * blockDim.x)
        if (!taken[g]) flist[frank[g]] = g;
}

__global__ void k_rg_assign(const int32_t *__restrict__ mark, const int32_t *__restrict__ corner,
                            const int32_t *__restrict__ child, int n, int PX, int PY, int ng,
                            const int32_t *__restrict__ flist, const int32_t *__restrict__ mrank,
                            const int32_t *__restrict__ n_moved, const int32_t *__restrict__ nrank,
                            int32_t *__restrict__ gnew, int32_t *__restrict__ gpar) {
    const int M = *n_moved;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        const int64_t p = pos_index(corner[3 * s] >> 3, corner[3 * s + 1] >> 3, corner[3 * s + 2] >> 3, PX, PY);
        const int og = child[s];
        if (!mark[p] || (og >= 0 && og < ng)) continue;
        const int g = flist[og >= 0 ? mrank[og] : M + nrank[p]];
        gnew[s] = g;
        gpar[g] = s;
    }
}

// The new level's tables, slot j = 8 g + k (k: x fastest): corner, parent,
// the old slot whose data moves here (-1: none -- the data is already in
// place, or is interpolated from the parent: job info in the GHOST_INFO
// layout of k_interp_patches, parent -1 for kept slots), child (the
// grandchildren of an old slot keep their group), new_of[old] = j.
__global__ void k_rg_new_slots(int nn, const int32_t *__restrict__ gpar, const int32_t *__restrict__ lcorner,
                               const int32_t *__restrict__ lchild_old, const int32_t *__restrict__ fchild_old,
                               int32_t *__restrict__ corner, int32_t *__restrict__ parent, int32_t *__restrict__ child,
                               int32_t *__restrict__ old_of, int32_t *__restrict__ info, int32_t *__restrict__ new_of) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nn; j += gridDim.x * blockDim.x) {
        const int g = j >> 3, k = j & 7, lx = k & 1, ly = (k >> 1) & 1, lz = k >> 2;
        const int P = gpar[g];
        corner[3 * j] = 2 * lcorner[3 * P] + 8 * lx;
        corner[3 * j + 1] = 2 * lcorner[3 * P + 1] + 8 * ly;
        corner[3 * j + 2] = 2 * lcorner[3 * P + 2] + 8 * lz;
        parent[j] = P;
        int32_t *I = info + (int64_t)GHOST_INFO * j;
        const int og = lchild_old[P];
        if (og >= 0) {
            const int o = 8 * og + k;
            old_of[j] = o == j ? -1 : o;
            child[j] = fchild_old[o];
            new_of[o] = j;
            I[0] = -1;
        } else {
            old_of[j] = -1;
            child[j] = -1;
            I[0] = P;
            I[1] = lx;
            I[2] = ly;
            I[3] = lz;
            I[4] = 8 << 12 | 8 << 16 | 8 << 20;  // the whole patch
        }
    }
}

// 26 siblings of every new slot from the level's position map (periodic)
__global__ void k_rg_sib(int nn, const int32_t *__restrict__ corner, const int32_t *__restrict__ posmap, int PX,
                         int PY, int PZ, int32_t *__restrict__ sib) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)nn * 26;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(i / 26), k = (int)(i % 26);
        const int kk = k + (k >= 13);  // skip the patch itself
        const int dx = kk % 3 - 1, dy = (kk / 3) % 3 - 1, dz = kk / 9 - 1;
        const int px = wrapd((corner[3 * j] >> 3) + dx, PX), py = wrapd((corner[3 * j + 1] >> 3) + dy, PY),
                  pz = wrapd((corner[3 * j + 2] >> 3) + dz, PZ);
        sib[i] = posmap[pos_index(px, py, pz, PX, PY)];
    }
}

__global__ void k_rg_commit(int n_l, const int32_t *__restrict__ gnew, int32_t *__restrict__ lchild, int n_g2,
                            int32_t *__restrict__ g2parent, const int32_t *__restrict__ new_of, int n_old,
                            int32_t *err) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int stride = gridDim.x * blockDim.x;
    for (int s = i; s < n_l; s += stride) lchild[s] = gnew[s];
    for (int y = i; y < n_g2; y += stride) {
        const int op = g2parent[y];
        const int np = (op >= 0 && op < n_old) ? new_of[op] : -1;
        if (np < 0) atomicOr(err, 1);
        else g2parent[y] = np;
    }
}

// ---- neighbour plan of a level (section 3.2 ghosts) --------------------------------

// Entry pos of group g's 4x4x4 source table (as build_nbr_plan on the host):
// a same-level slot, or a coarse-fine ghost patch, first recorded as
// -2 - (its patch-position index) with the cells any group reads OR-ed into
// gbits (per dimension: bit "low bound 0" and bit "high bound 8", plus a
// presence bit), or -1 for a corner position no stencil reads.
__global__ void k_plan_nbr(int n_groups, const int32_t *__restrict__ corner, const int32_t *__restrict__ sib, int PX,
                           int PY, int PZ, int corners, int32_t *__restrict__ nbr, int32_t *__restrict__ gbits,
                           int32_t *err) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)n_groups * 64;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int g = (int)(i >> 6), pos = (int)(i & 63);
        const int q3[3] = {(pos & 3) - 1, ((pos >> 2) & 3) - 1, (pos >> 4) - 1};
        int p3[3], d3[3];
        for (int d = 0; d < 3; d++) {
            p3[d] = q3[d] < 0 ? 0 : (q3[d] > 1 ? 1 : q3[d]);
            d3[d] = q3[d] - p3[d];
        }
        const int own = 8 * g + p3[0] + 2 * p3[1] + 4 * p3[2];
        if (!d3[0] && !d3[1] && !d3[2]) {
            nbr[i] = own;
            continue;
        }
        const int32_t s = sib[(int64_t)own * 26 + sib_kd(d3[0], d3[1], d3[2])];
        if (s >= 0) {
            nbr[i] = s;
            continue;
        }
        const bool corner_pos = d3[0] && d3[1] && d3[2];
        if (corner_pos && !corners) {
            nbr[i] = -1;
            continue;
        }
        const int px = wrapd((corner[3 * own] >> 3) + d3[0], PX), py = wrapd((corner[3 * own + 1] >> 3) + d3[1], PY),
                  pz = wrapd((corner[3 * own + 2] >> 3) + d3[2], PZ);
        const int64_t p = pos_index(px, py, pz, PX, PY);
        int bits = 1 << 6;
        for (int d = 0; d < 3; d++) {
            if (q3[d] >= 0) bits |= 1 << d;        // low bound 0 (else 8 - depth)
            if (q3[d] <= 1) bits |= 1 << (3 + d);  // high bound 8 (else depth)
        }
        atomicOr(gbits + p, bits);
        nbr[i] = (int32_t)(-2 - p);
    }
}

// ghost patch id -> job of k_interp_patches: the coarse patch holding it and
// its position inside that patch's children (0/1 per dimension), the box of
// cells read
__global__ void k_plan_ghosts(int64_t npos, const int32_t *__restrict__ gbits, const int32_t *__restrict__ grank,
                              const int32_t *__restrict__ posmap_c, int PX, int PY, int depth,
                              int32_t *__restrict__ info, int cap, int32_t *err) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < npos; p += (int64_t)gridDim.x * blockDim.x) {
        const int b = gbits[p];
        if (!b) continue;
        const int id = grank[p];
        if (id >= cap) {
            atomicOr(err, 2);
            continue;
        }
        const int px = (int)(p % PX), py = (int)((p / PX) % PY), pz = (int)(p / ((int64_t)PX * PY));
        const int32_t cp = posmap_c[pos_index(px >> 1, py >> 1, pz >> 1, PX >> 1, PY >> 1)];
        if (cp < 0) atomicOr(err, 1);
        int box = 0;
        for (int d = 0; d < 3; d++) {
            const int lo = (b >> d) & 1 ? 0 : 8 - depth, hi = (b >> (3 + d)) & 1 ? 8 : depth;
            box |= lo << (4 * d) | hi << (12 + 4 * d);
        }
        int32_t *I = info + (int64_t)GHOST_INFO * id;
        I[0] = cp;
        I[1] = px & 1;
        I[2] = py & 1;
        I[3] = pz & 1;
        I[4] = box;
    }
}

// VL on refined levels: the 27 patch positions around each ghost patch
// (a slot of the level, another ghost patch as -2 - id, or -1)
__global__ void k_plan_ghost_nbr(int64_t npos, const int32_t *__restrict__ gbits, const int32_t *__restrict__ grank,
                                 const int32_t *__restrict__ posmap, int PX, int PY, int PZ, int cap,
                                 int32_t *__restrict__ gnbr) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < npos; p += (int64_t)gridDim.x * blockDim.x) {
        if (!gbits[p]) continue;
        const int id = grank[p];
        if (id >= cap) continue;
        const int px = (int)(p % PX), py = (int)((p / PX) % PY), pz = (int)(p / ((int64_t)PX * PY));
        for (int k = 0; k < 27; k++) {
            const int qx = wrapd(px + k % 3 - 1, PX), qy = wrapd(py + (k / 3) % 3 - 1, PY),
                      qz = wrapd(pz + k / 9 - 1, PZ);
            const int64_t q = pos_index(qx, qy, qz, PX, PY);
            const int32_t s = posmap[q];
            gnbr[(int64_t)id * 27 + k] = s >= 0 ? s : (gbits[q] ? -2 - grank[q] : -1);
        }
    }
}

__global__ void k_plan_fix(int64_t n, int32_t *__restrict__ nbr, const int32_t *__restrict__ grank) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = nbr[i];
        if (v <= -2) nbr[i] = -2 - grank[-2 - (int64_t)v];
    }
}

// ---- coarse-fine register maps (section 2.2) ------------------------------------------

// fine side: group face f of fine group g lies on an interface when the
// coarse neighbour of its parent across f is a leaf
__global__ void k_cf_fine_flags(int n_groups_f, const int32_t *__restrict__ fparent, const int32_t *__restrict__ csib,
                                const int32_t *__restrict__ cchild, int n_c, int32_t *__restrict__ flag, int32_t *err) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_groups_f * 6; i += gridDim.x * blockDim.x) {
        const int g = i / 6, f = i % 6;
        const int P = fparent[8 * g];
        int fl = 0;
        if (P < 0 || P >= n_c) {
            atomicOr(err, 1);
        } else {
            const int Q = csib[(int64_t)P * 26 + face_sib_d(f)];
            if (Q < 0) atomicOr(err, 1);
            else fl = cchild[Q] < 0;
        }
        flag[i] = fl;
    }
}

__global__ void k_cf_fine_off(int n, const int32_t *__restrict__ flag, const int32_t *__restrict__ rank,
                              int64_t block, int64_t *__restrict__ fine_off) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        fine_off[i] = flag[i] ? (int64_t)rank[i] * block : -1;
}

// coarse side: per coarse patch Q, register flags of its faces (leaf Q next to
// a refined P), whether it needs a fix-up entry, whether it is restricted
__global__ void k_cf_coarse_flags(int n_c, const int32_t *__restrict__ csib, const int32_t *__restrict__ cchild,
                                  int32_t *__restrict__ fflag, int32_t *__restrict__ fix, int32_t *__restrict__ rst) {
    for (int Q = blockIdx.x * blockDim.x + threadIdx.x; Q < n_c; Q += gridDim.x * blockDim.x) {
        int any = 0;
        const bool refined = cchild[Q] >= 0;
        for (int f = 0; f < 6; f++) {
            int fl = 0;
            if (!refined) {
                const int P = csib[(int64_t)Q * 26 + face_sib_d(f)];
                fl = P >= 0 && cchild[P] >= 0;
            }
            fflag[Q * 6 + f] = fl;
            any |= fl;
        }
        fix[Q] = any;
        rst[Q] = refined;
    }
}

__global__ void k_cf_coarse_write(int n_c, const int32_t *__restrict__ csib, const int32_t *__restrict__ cchild,
                                  const int32_t *__restrict__ fflag, const int32_t *__restrict__ frank,
                                  const int32_t *__restrict__ fix, const int32_t *__restrict__ fixrank,
                                  const int32_t *__restrict__ rst, const int32_t *__restrict__ rstrank,
                                  const int64_t *__restrict__ fine_off, int64_t cblock, int64_t *__restrict__ coarse_off,
                                  int64_t *__restrict__ fix_list, int32_t *__restrict__ restrict_list, int32_t *err) {
    for (int Q = blockIdx.x * blockDim.x + threadIdx.x; Q < n_c; Q += gridDim.x * blockDim.x) {
        if (rst[Q]) {
            const int r = rstrank[Q];
            restrict_list[2 * r] = Q;
            restrict_list[2 * r + 1] = cchild[Q];
        }
        int64_t e[13];
        e[0] = Q;
        for (int f = 0; f < 6; f++) {
            int64_t co = -1, fo = -1;
            if (fflag[Q * 6 + f]) {
                co = (int64_t)frank[Q * 6 + f] * cblock;
                const int P = csib[(int64_t)Q * 26 + face_sib_d(f)];
                fo = fine_off[(int64_t)cchild[P] * 6 + (f ^ 1)];
                if (fo < 0) atomicOr(err, 1);
            }
            coarse_off[Q * 6 + f] = co;
            e[1 + f] = co;
            e[7 + f] = fo;
        }
        if (fix[Q]) {
            int64_t *o = fix_list + (int64_t)fixrank[Q] * 13;
            for (int k = 0; k < 13; k++) o[k] = e[k];
        }
    }
}

// ---- z-runs of a refined level (the counterpart of z_chains, choose_run_len
// and cut_runs of the host plan: the same chains, length and runs, closed
// cycles listed among the open chains by their head) ----
//
// Group u is g's upper neighbour when position (1,1,3) of g's 4x4x4 table
// (index 53) holds u's first patch and position (1,1,0) of u (index 5) holds
// g's patch (0,0,1): same-level groups stacked in z.  The relation is one to
// one.
__global__ void k_run_links(int ng, const int32_t *__restrict__ nbr, int32_t *__restrict__ up,
                            int32_t *__restrict__ down) {
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < ng; g += gridDim.x * blockDim.x) {
        const int32_t s = nbr[(int64_t)g * 64 + 53];
        int u = -1;
        if (s >= 0 && s % 8 == 0) {
            const int cand = s / 8;
            if (cand != g && cand < ng && nbr[(int64_t)cand * 64 + 5] == 8 * g + 4) u = cand;
        }
        up[g] = u;
        if (u >= 0) down[u] = g;
    }
}

// Chain heads and their lengths (0 elsewhere), with a histogram of the
// lengths (bins 1..hmax, longer ones in bin hmax): a group with no lower
// neighbour heads the chain of upper neighbours above it; a closed cycle (a
// periodic column) is headed by its lowest group id.  Walks are bounded by
// the group count.
__global__ void k_run_heads(int ng, const int32_t *__restrict__ up, const int32_t *__restrict__ down,
                            int32_t *__restrict__ clen, int32_t *__restrict__ hist, int hmax) {
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < ng; g += gridDim.x * blockDim.x) {
        int L = 0;
        if (down[g] < 0) {
            L = 1;
            for (int x = up[g]; x >= 0 && L < ng; x = up[x]) L++;
        } else {
            int x = up[g], m = g, n = 1;
            while (x >= 0 && x != g && n < ng) {
                m = x < m ? x : m;
                x = up[x];
                n++;
            }
            if (x == g && m == g) L = n;
        }
        clen[g] = L;
        if (L) atomicAdd(hist + (L < hmax ? L : hmax), 1);
    }
}

// The run length in 1..32 minimising the round-robin estimate
// ceil(n_runs / grid) (min(len, longest) + e), from the length histogram
// (one block; the first minimum, as on the host); out[0] = the number of
// runs of that length, out[1] = the length.
constexpr int RUN_NT = 256, RUN_MAXLEN = 32;
__global__ void __launch_bounds__(RUN_NT) k_run_len(const int32_t *__restrict__ hist, int hmax, int grid, double e,
                                                    int32_t *__restrict__ out) {
    __shared__ unsigned long long cnt[RUN_MAXLEN];
    __shared__ double cost[RUN_MAXLEN];
    __shared__ int longest;
    if (threadIdx.x < RUN_MAXLEN) cnt[threadIdx.x] = 0ull;
    if (threadIdx.x == 0) longest = 0;
    __syncthreads();
    for (int L = 1 + threadIdx.x; L <= hmax; L += RUN_NT) {
        const unsigned long long h = (unsigned)hist[L];
        if (!h) continue;
        atomicMax(&longest, L);
#pragma unroll
        for (int k = 0; k < RUN_MAXLEN; k++) atomicAdd(&cnt[k], h * (unsigned)((L + k) / (k + 1)));
    }
    __syncthreads();
    if (threadIdx.x < RUN_MAXLEN) {
        const int len = threadIdx.x + 1;
        const long long rounds = ((long long)cnt[threadIdx.x] + grid - 1) / grid;
        cost[threadIdx.x] = (double)rounds * ((len < longest ? len : longest) + e);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int best_len = 1;
        double best = 1e300;
        for (int k = 0; k < RUN_MAXLEN; k++)
            if (cost[k] < best - 1e-9) {
                best = cost[k];
                best_len = k + 1;
            }
        out[0] = (int32_t)cnt[best_len - 1];
        out[1] = best_len;
    }
}

// Runs per chain head for the chosen length.
__global__ void k_run_count(int ng, const int32_t *__restrict__ clen, const int32_t *__restrict__ lenp,
                            int32_t *__restrict__ rcnt) {
    const int len = *lenp;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < ng; g += gridDim.x * blockDim.x)
        rcnt[g] = (clen[g] + len - 1) / len;
}

// Each head writes its chain at lpos and its runs' offsets at rpos; the
// head whose runs come last also closes run_off.
__global__ void k_run_write(int ng, const int32_t *__restrict__ up, const int32_t *__restrict__ clen,
                            const int32_t *__restrict__ lpos, const int32_t *__restrict__ rpos,
                            const int32_t *__restrict__ lenp, const int32_t *__restrict__ n_runs,
                            int32_t *__restrict__ runs, int32_t *__restrict__ run_off) {
    const int len = *lenp, total = *n_runs;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < ng; g += gridDim.x * blockDim.x) {
        const int L = clen[g];
        if (!L) continue;
        const int a = lpos[g], r0 = rpos[g], R = (L + len - 1) / len;
        int x = g;
        for (int i = 0; i < L; i++) {
            runs[a + i] = x;
            x = up[x];
        }
        for (int r = 0; r < R; r++) run_off[r0 + r] = a + r * len;
        if (r0 + R == total) run_off[total] = a + L;
    }
}

inline int grid_for(int64_t n, int nt, int cap) {
    const int64_t b = (n + nt - 1) / nt;
    return (int)(b < 1 ? 1 : (b < cap ? b : cap));
}

}  // namespace

// Exclusive scan of n int32 values into out; the total goes to *total (device).
static amr_status scan_i32(amr_hydro_ctx *c, const int32_t *in, int32_t *out, int64_t n, int32_t *total, int flags) {
    amr_status st;
    const int nb = (int)((n + SCAN_BLOCK - 1) / SCAN_BLOCK);
    if ((st = c->rg.bsum.reserve(nb > 0 ? nb : 1))) return st;
    if (n == 0) return cuda_fail(cudaMemsetAsync(total, 0, 4, c->stream), "memset");
    k_scan_block<<<nb, SCAN_NT, 0, c->stream>>>(in, out, c->rg.bsum.p, (int)n, flags, total);
    if (nb == 1) return cuda_fail(cudaGetLastError(), "scan");
    k_scan_sums<<<1, SCAN_NT, 0, c->stream>>>(c->rg.bsum.p, nb, total);
    k_scan_add<<<(int)((n + 255) / 256), 256, 0, c->stream>>>(out, c->rg.bsum.p, (int)n);
    return cuda_fail(cudaGetLastError(), "scan");
}

static void patch_grid(const amr_hydro_ctx *c, int level, int P[3]) {
    for (int d = 0; d < 3; d++) P[d] = (c->prm.root_n[d] << level) / 8;
}

// The dense position -> slot map of a level from its device corner table.
amr_status build_posmap(amr_hydro_ctx *c, int level) {
    Level &L = c->lv[level];
    int P[3];
    patch_grid(c, level, P);
    const int64_t np = (int64_t)P[0] * P[1] * P[2];
    amr_status st;
    if ((st = L.posmap.reserve(np))) return st;
    if ((st = cuda_fail(cudaMemsetAsync(L.posmap.p, 0xff, 4 * np, c->stream), "memset posmap"))) return st;
    if (L.n_patches) {
        k_posmap_scatter<<<grid_for(L.n_patches, 256, 4 * c->n_sm), 256, 0, c->stream>>>(L.posmap.p, L.d_corner,
                                                                                       L.n_patches, P[0], P[1]);
        if ((st = cuda_fail(cudaGetLastError(), "k_posmap_scatter"))) return st;
    }
    L.posmap_valid = true;
    return AMR_OK;
}

// Neighbour plan of level X >= 1 on the device (the counterpart of
// build_nbr_plan + plan_level on the host; its z-runs: plan_runs_dev).  Queues the
// kernels; the ghost count lands in *n_ghost_dev.
// z-runs of level X from its neighbour plan: the chains and the run length
// (run_cnt[0] = the number of runs, run_cnt[1] = their length); the runs
// themselves (L.runs / L.run_off, plan_runs_write) only when the length
// exceeds 1, as the host plan does.
static amr_status plan_runs_dev(amr_hydro_ctx *c, int X, int32_t *run_cnt) {
    Level &L = c->lv[X];
    auto &S = c->rg;
    const int ng = L.n_groups;
    amr_status st;
    // the chains stay with the level until plan_runs_write (another level's
    // plan may run in between)
    if ((st = L.chain_up.reserve(ng + 1)) || (st = S.run_down.reserve(ng + 1)) || (st = L.chain_len.reserve(ng + 1)))
        return st;
    // a chain holds at most the level's column of groups
    const int hmax = ((c->prm.root_n[2] << X) + 15) / 16;
    if ((st = S.run_hist.reserve(hmax + 1))) return st;
    if ((st = cuda_fail(cudaMemsetAsync(S.run_down.p, 0xff, 4 * (size_t)ng, c->stream), "memset")) ||
        (st = cuda_fail(cudaMemsetAsync(S.run_hist.p, 0, 4 * (size_t)(hmax + 1), c->stream), "memset")))
        return st;
    const int gb = grid_for(ng, 256, 8 * c->n_sm);
    k_run_links<<<gb, 256, 0, c->stream>>>(ng, L.nbr.p, L.chain_up.p, S.run_down.p);
    k_run_heads<<<gb, 256, 0, c->stream>>>(ng, L.chain_up.p, S.run_down.p, L.chain_len.p, S.run_hist.p, hmax);
    k_run_len<<<1, RUN_NT, 0, c->stream>>>(S.run_hist.p, hmax, c->n_sm * c->step_bps,
                                           c->prm.prec == AMR_FP64 ? 0.05 : 0.13, run_cnt);
    return cuda_fail(cudaGetLastError(), "z-runs");
}

// The runs of plan_runs_dev's chains and length (after the host read the
// counts: queued only when the length exceeds 1).
static amr_status plan_runs_write(amr_hydro_ctx *c, int X, int32_t *run_cnt) {
    Level &L = c->lv[X];
    auto &S = c->rg;
    const int ng = L.n_groups;
    amr_status st;
    if ((st = S.run_cnt.reserve(ng + 1)) || (st = S.run_lpos.reserve(ng + 1)) || (st = S.run_rpos.reserve(ng + 1)) ||
        (st = L.runs.reserve(ng + 1)) || (st = L.run_off.reserve(ng + 2)))
        return st;
    const int gb = grid_for(ng, 256, 8 * c->n_sm);
    k_run_count<<<gb, 256, 0, c->stream>>>(ng, L.chain_len.p, run_cnt + 1, S.run_cnt.p);
    if ((st = cuda_fail(cudaGetLastError(), "k_run_count"))) return st;
    if ((st = scan_i32(c, L.chain_len.p, S.run_lpos.p, ng, run_cnt + 2, 0)) ||
        (st = scan_i32(c, S.run_cnt.p, S.run_rpos.p, ng, run_cnt, 0)))
        return st;
    k_run_write<<<gb, 256, 0, c->stream>>>(ng, L.chain_up.p, L.chain_len.p, S.run_lpos.p, S.run_rpos.p, run_cnt + 1,
                                           run_cnt, L.runs.p, L.run_off.p);
    return cuda_fail(cudaGetLastError(), "k_run_write");
}

static amr_status plan_level_dev(amr_hydro_ctx *c, int X, int32_t *n_ghost_dev, int32_t *err) {
    Level &L = c->lv[X], &C = c->lv[X - 1];
    amr_status st;
    int P[3];
    patch_grid(c, X, P);
    const int64_t np = (int64_t)P[0] * P[1] * P[2];
    // ghost cells a step reads: two (PLM), three (PPM; the VL predictor's
    // half step on the two the corrector reads), in boxes of even depth
    const bool vl = c->prm.scheme == AMR_SCHEME_VL;
    const int depth = (c->prm.recon == AMR_RECON_PPM || vl) ? 4 : 2;
    L.n_runs = 0;
    if ((st = L.nbr.reserve((size_t)L.n_groups * 64 + 64))) return st;
    if ((st = L.gbits.reserve(np)) || (st = L.grank.reserve(np))) return st;
    // at most 56 ghost positions around a group
    const int cap = L.n_groups * 56 + 1;
    if ((st = L.ghost_info.reserve((size_t)cap * GHOST_INFO))) return st;
    if ((st = cuda_fail(cudaMemsetAsync(L.gbits.p, 0, 4 * np, c->stream), "memset"))) return st;
    if (!C.posmap_valid && (st = build_posmap(c, X - 1))) return st;
    const int64_t ne = (int64_t)L.n_groups * 64;
    k_plan_nbr<<<grid_for(ne, 256, 8 * c->n_sm), 256, 0, c->stream>>>(L.n_groups, L.d_corner, L.d_sib, P[0], P[1],
                                                                     P[2], c->prm.fallback != 0, L.nbr.p,
                                                                     L.gbits.p, err);
    if ((st = cuda_fail(cudaGetLastError(), "k_plan_nbr"))) return st;
    if ((st = scan_i32(c, L.gbits.p, L.grank.p, np, n_ghost_dev, true))) return st;
    k_plan_ghosts<<<grid_for(np, 256, 8 * c->n_sm), 256, 0, c->stream>>>(np, L.gbits.p, L.grank.p, C.posmap.p, P[0],
                                                                        P[1], depth, L.ghost_info.p, cap, err);
    if ((st = cuda_fail(cudaGetLastError(), "k_plan_ghosts"))) return st;
    if (vl) {
        if (!L.posmap_valid && (st = build_posmap(c, X))) return st;
        if ((st = L.ghost_nbr.reserve((size_t)cap * 27))) return st;
        k_plan_ghost_nbr<<<grid_for(np, 256, 8 * c->n_sm), 256, 0, c->stream>>>(np, L.gbits.p, L.grank.p, L.posmap.p,
                                                                                P[0], P[1], P[2], cap, L.ghost_nbr.p);
        if ((st = cuda_fail(cudaGetLastError(), "k_plan_ghost_nbr"))) return st;
    }
    k_plan_fix<<<grid_for(ne, 256, 8 * c->n_sm), 256, 0, c->stream>>>(ne, L.nbr.p, L.grank.p);
    L.plan_version++;
    return cuda_fail(cudaGetLastError(), "k_plan_fix");
}

// Coarse-fine register maps between level F >= 1 and its coarse level on
// the device (the counterpart of rebuild_cf); counts into cnt[0..3]
// (fine registers, coarse registers, fix-up entries, restrictions).
static amr_status cf_dev(amr_hydro_ctx *c, int F_, int32_t *cnt, int32_t *err) {
    Level &C = c->lv[F_ - 1], &F = c->lv[F_];
    amr_status st;
    const int nfg = F.n_groups * 6, nc = C.n_patches;
    if ((st = F.fine_off.reserve(nfg + 6)) || (st = C.coarse_off.reserve((size_t)nc * 6 + 6)) ||
        (st = C.fix_list.reserve((size_t)nc * 13 + 13)) || (st = C.restrict_list.reserve((size_t)nc * 2 + 2)))
        return st;
    auto &S = c->rg;
    if ((st = S.cf_a.reserve(nfg + 1)) || (st = S.cf_b.reserve(nfg + 1)) ||
        (st = S.cf_c.reserve((size_t)nc * 6 + 1)) || (st = S.cf_d.reserve((size_t)nc * 6 + 1)) ||
        (st = S.cf_e.reserve(nc + 1)) || (st = S.cf_f.reserve(nc + 1)) || (st = S.cf_g.reserve(nc + 1)) ||
        (st = S.cf_h.reserve(nc + 1)))
        return st;
    if (nfg) {
        k_cf_fine_flags<<<grid_for(nfg, 256, 8 * c->n_sm), 256, 0, c->stream>>>(F.n_groups, F.d_parent, C.d_sib,
                                                                               C.d_child, nc, S.cf_a.p, err);
        if ((st = scan_i32(c, S.cf_a.p, S.cf_b.p, nfg, cnt + 0, false))) return st;
        k_cf_fine_off<<<grid_for(nfg, 256, 8 * c->n_sm), 256, 0, c->stream>>>(nfg, S.cf_a.p, S.cf_b.p, fine_block(c),
                                                                             F.fine_off.p);
    } else if ((st = cuda_fail(cudaMemsetAsync(cnt + 0, 0, 4, c->stream), "memset"))) {
        return st;
    }
    if (nc) {
        k_cf_coarse_flags<<<grid_for(nc, 256, 8 * c->n_sm), 256, 0, c->stream>>>(nc, C.d_sib, C.d_child, S.cf_c.p,
                                                                                S.cf_e.p, S.cf_g.p);
        if ((st = scan_i32(c, S.cf_c.p, S.cf_d.p, (int64_t)nc * 6, cnt + 1, false)) ||
            (st = scan_i32(c, S.cf_e.p, S.cf_f.p, nc, cnt + 2, false)) ||
            (st = scan_i32(c, S.cf_g.p, S.cf_h.p, nc, cnt + 3, false)))
            return st;
        k_cf_coarse_write<<<grid_for(nc, 256, 8 * c->n_sm), 256, 0, c->stream>>>(
            nc, C.d_sib, C.d_child, S.cf_c.p, S.cf_d.p, S.cf_e.p, S.cf_f.p, S.cf_g.p, S.cf_h.p, F.fine_off.p,
            coarse_block(c), C.coarse_off.p, C.fix_list.p, C.restrict_list.p, err);
    }
    return cuda_fail(cudaGetLastError(), "cf maps");
}

// After the counts arrived on the host: sizes, register buffers.
static amr_status cf_finish(amr_hydro_ctx *c, int F_, const int32_t *cnt) {
    Level &C = c->lv[F_ - 1], &F = c->lv[F_];
    amr_status st;
    const int nf = cnt[0], nc = cnt[1];
    if (nf && (st = F.freg.reserve((size_t)nf * fine_block(c)))) return st;
    if (nc && (st = C.creg.reserve((size_t)nc * coarse_block(c)))) return st;
    if (nf && (st = cuda_fail(cudaMemsetAsync(F.freg.p, 0, sizeof(double) * fine_block(c) * (size_t)nf, c->stream),
                              "memset")))
        return st;
    F.n_freg = nf;
    C.n_creg = nc;
    C.n_fix = cnt[2];
    C.n_restrict = cnt[3];
    return AMR_OK;
}

static amr_status read_counts(amr_hydro_ctx *c, int n) {
    amr_status st = cuda_fail(cudaMemcpyAsync(c->rg.hcnt, c->rg.cnt.p, 4 * n, cudaMemcpyDeviceToHost, c->stream),
                              "d2h counts");
    if (st) return st;
    return cuda_fail(cudaStreamSynchronize(c->stream), "sync");
}

// Regrid of level l (section 2.1) on the device: rebuilds level l+1.
amr_status regrid_dev(amr_hydro_ctx *c, int l) {
    Level &L = c->lv[l], &F = c->lv[l + 1];
    Level *G2 = (l + 2 <= c->prm.lmax && c->lv[l + 2].n_patches) ? &c->lv[l + 2] : nullptr;
    auto &S = c->rg;
    amr_status st;
    const int n = L.n_patches;
    int PL[3], PF[3];
    patch_grid(c, l, PL);
    patch_grid(c, l + 1, PF);
    const int64_t npl = (int64_t)PL[0] * PL[1] * PL[2];
    if ((st = S.cnt.reserve(32))) return st;
    int32_t *cnt = S.cnt.p;
    if ((st = cuda_fail(cudaMemsetAsync(cnt, 0, 4 * 32, c->stream), "memset"))) return st;
    // refinement flags (cell criterion + flag buffer)
    if ((st = c->pflag.reserve(n))) return st;
    if ((st = patch_flags_dev(c, l, c->pflag.p))) return st;
    if (!L.posmap_valid && (st = build_posmap(c, l))) return st;
    if ((st = S.keep.reserve(n + 1)) || (st = S.mark.reserve(npl)) || (st = S.rank.reserve(npl)) ||
        (st = S.gnew.reserve(n + 1)) || (st = S.gpar.reserve(n + 1)))
        return st;
    const int gl = grid_for(n, 256, 8 * c->n_sm);
    if (G2) {
        if ((st = cuda_fail(cudaMemsetAsync(S.keep.p, 0, 4 * (size_t)n, c->stream), "memset"))) return st;
        k_rg_keep<<<grid_for(F.n_patches, 128, 8 * c->n_sm), 128, 0, c->stream>>>(
            F.d_corner, F.d_child, F.n_patches, L.posmap.p, PL[0], PL[1], PL[2], S.keep.p, cnt + 0);
        if ((st = cuda_fail(cudaGetLastError(), "k_rg_keep"))) return st;
    }
    if ((st = cuda_fail(cudaMemsetAsync(S.mark.p, 0, 4 * npl, c->stream), "memset"))) return st;
    k_rg_select<<<gl, 256, 0, c->stream>>>(c->pflag.p, L.d_sib, L.d_child, G2 ? S.keep.p : nullptr, L.d_corner, n,
                                           PL[0], PL[1], S.mark.p);
    if ((st = cuda_fail(cudaGetLastError(), "k_rg_select"))) return st;
    k_rg_classify<<<gl, 256, 0, c->stream>>>(S.mark.p, L.d_corner, L.d_child, n, PL[0], PL[1], cnt + 1, cnt + 2);
    if ((st = cuda_fail(cudaGetLastError(), "k_rg_classify"))) return st;
    if ((st = read_counts(c, 3))) return st;
    if (S.hcnt[0]) return AMR_E_NESTING;
    if (!S.hcnt[1]) return AMR_OK;  // the refined set is unchanged
    const int ng = S.hcnt[2], nn = 8 * ng;
    if (nn > c->prm.max_patches) return AMR_E_NOMEM;

    // group numbers, slots kept in place (k_rg_keepmark); counts of free
    // numbers, moved and new groups into cnt[21..23]
    const int ng_old = F.n_groups;
    if ((st = S.taken.reserve(ng + 1)) || (st = S.frank.reserve(ng + 1)) || (st = S.flist.reserve(ng + 1)) ||
        (st = S.mflag.reserve(ng_old + 1)) || (st = S.mrank.reserve(ng_old + 1)) || (st = S.nflag.reserve(npl)))
        return st;
    if ((st = cuda_fail(cudaMemsetAsync(S.taken.p, 0, 4 * ((size_t)ng + 1), c->stream), "memset")) ||
        (st = cuda_fail(cudaMemsetAsync(S.mflag.p, 0, 4 * ((size_t)ng_old + 1), c->stream), "memset")) ||
        (st = cuda_fail(cudaMemsetAsync(S.nflag.p, 0, 4 * (size_t)npl, c->stream), "memset")))
        return st;
    k_rg_keepmark<<<gl, 256, 0, c->stream>>>(S.mark.p, L.d_corner, L.d_child, n, PL[0], PL[1], ng, S.gnew.p, S.gpar.p,
                                             S.taken.p, S.mflag.p, S.nflag.p);
    if ((st = cuda_fail(cudaGetLastError(), "k_rg_keepmark"))) return st;
    if ((st = scan_i32(c, S.taken.p, S.frank.p, ng, cnt + 21, 2)) ||
        (st = scan_i32(c, S.mflag.p, S.mrank.p, ng_old, cnt + 22, 0)) ||
        (st = scan_i32(c, S.nflag.p, S.rank.p, npl, cnt + 23, 0)))
        return st;
    k_rg_freelist<<<grid_for(ng, 256, 8 * c->n_sm), 256, 0, c->stream>>>(ng, S.taken.p, S.frank.p, S.flist.p);
    k_rg_assign<<<gl, 256, 0, c->stream>>>(S.mark.p, L.d_corner, L.d_child, n, PL[0], PL[1], ng, S.flist.p, S.mrank.p,
                                           cnt + 22, S.rank.p, S.gnew.p, S.gpar.p);
    // the step's work list: the groups in position order (nflag's buffer
    // takes the chosen positions' ranks)
    if ((st = F.work.reserve(ng + 1))) return st;
    if ((st = scan_i32(c, S.mark.p, S.nflag.p, npl, cnt + 24, 0))) return st;
    k_rg_order<<<gl, 256, 0, c->stream>>>(S.mark.p, S.nflag.p, L.d_corner, S.gnew.p, n, PL[0], PL[1], F.work.p);
    F.has_work = true;
    if ((st = cuda_fail(cudaGetLastError(), "k_rg_assign"))) return st;

    // the new level's tables (into scratch first: the old ones are still read)
    const int n_old = F.n_patches;
    if ((st = S.corner.reserve((size_t)nn * 3 + 3)) || (st = S.sib.reserve((size_t)nn * 26 + 26)) ||
        (st = S.parent.reserve(nn + 1)) || (st = S.child.reserve(nn + 1)) || (st = S.old_of.reserve(nn + 1)) ||
        (st = S.info.reserve((size_t)nn * GHOST_INFO + GHOST_INFO)) || (st = S.new_of.reserve(n_old + 1)))
        return st;
    if ((st = cuda_fail(cudaMemsetAsync(S.new_of.p, 0xff, 4 * ((size_t)n_old + 1), c->stream), "memset"))) return st;
    if (nn) {
        k_rg_new_slots<<<grid_for(nn, 256, 8 * c->n_sm), 256, 0, c->stream>>>(
            nn, S.gpar.p, L.d_corner, L.d_child, F.d_child, S.corner.p, S.parent.p, S.child.p, S.old_of.p, S.info.p,
            S.new_of.p);
        if ((st = cuda_fail(cudaGetLastError(), "k_rg_new_slots"))) return st;
    }
    // cell data of the new level in place (with dual energy also the
    // entropy): kept groups stay in their slots, moved ones are copied from
    // slots >= nn into free slots < nn, new ones are interpolated into the
    // remaining free slots
    double *Ud = F.U[F.cur];
    const bool de = c->prm.dual_energy != 0;
    if (de && (!F.S[0] || !F.S[1] || !L.S[0])) return AMR_E_INVAL;  // amr_hydro_set_entropy first
    if (n_old && nn && (st = copy_slots(c, Ud, Ud, S.old_of.p, nn))) return st;
    if (de && n_old && nn && (st = copy_slots(c, F.S[F.cur], F.S[F.cur], S.old_of.p, nn, PV))) return st;
    if ((st = interp_new_patches(c, l, Ud, nullptr, S.info.p, nn, de ? F.S[F.cur] : nullptr))) return st;
    // commit: level l's child groups, grandchildren's parents, the new tables
    const int n_g2 = G2 ? G2->n_patches : 0;
    k_rg_commit<<<grid_for(n > n_g2 ? n : n_g2, 256, 8 * c->n_sm), 256, 0, c->stream>>>(
        n, S.gnew.p, L.w_child, n_g2, G2 ? G2->w_parent : nullptr, S.new_of.p, n_old, cnt + 0);
    if ((st = cuda_fail(cudaGetLastError(), "k_rg_commit"))) return st;
    if (nn) {
        if ((st = cuda_fail(cudaMemcpyAsync(F.w_corner, S.corner.p, 12 * (size_t)nn, cudaMemcpyDeviceToDevice,
                                            c->stream), "d2d")) ||
            (st = cuda_fail(cudaMemcpyAsync(F.w_parent, S.parent.p, 4 * (size_t)nn, cudaMemcpyDeviceToDevice,
                                            c->stream), "d2d")) ||
            (st = cuda_fail(cudaMemcpyAsync(F.w_child, S.child.p, 4 * (size_t)nn, cudaMemcpyDeviceToDevice,
                                            c->stream), "d2d")))
            return st;
    }
    F.n_patches = nn;
    F.n_groups = ng;
    F.t = F.t_prev = L.t;
    F.t_pending = false;
    F.speed_valid = false;
    F.ring = 0;
    F.host_stale = L.host_stale = true;
    if (G2) G2->host_stale = true;
    F.version++;
    F.structure++;
    if ((st = build_posmap(c, l + 1))) return st;
    if (nn) {
        k_rg_sib<<<grid_for((int64_t)nn * 26, 256, 8 * c->n_sm), 256, 0, c->stream>>>(nn, F.d_corner, F.posmap.p,
                                                                                      PF[0], PF[1], PF[2], F.w_sib);
        if ((st = cuda_fail(cudaGetLastError(), "k_rg_sib"))) return st;
    }
    {
        const double rec[3] = {0.0, F.t, F.t};
        std::memcpy(S.htime, rec, 24);
        if ((st = cuda_fail(cudaMemcpyAsync(c->dtbuf.p + 3 * (l + 1), S.htime, 24, cudaMemcpyHostToDevice, c->stream),
                            "h2d time")))
            return st;
    }
    if ((st = cuda_fail(cudaMemsetAsync(c->scal.p + F.scal0, 0, 8 * SCAL_PER, c->stream), "memset"))) return st;
    if (!ng) F.dt_prev = -1.0;
    // plans and register maps of the changed levels; one read of their counts
    L.n_creg = L.n_fix = L.n_restrict = 0;
    F.n_ghost = F.n_freg = 0;
    F.n_creg = F.n_fix = F.n_restrict = 0;
    if (nn) {
        if ((st = plan_level_dev(c, l + 1, cnt + 4, cnt + 0))) return st;
        if ((st = plan_runs_dev(c, l + 1, cnt + 14))) return st;
        if ((st = cf_dev(c, l + 1, cnt + 5, cnt + 0))) return st;
        if (G2) {
            if ((st = plan_level_dev(c, l + 2, cnt + 9, cnt + 0))) return st;
            if ((st = plan_runs_dev(c, l + 2, cnt + 17))) return st;
            if ((st = cf_dev(c, l + 2, cnt + 10, cnt + 0))) return st;
        }
    }
    if ((st = read_counts(c, 20))) return st;
    if (S.hcnt[0] & 2) return AMR_E_NOMEM;
    if (S.hcnt[0]) return AMR_E_NESTING;
    if (nn) {
        F.n_runs = S.hcnt[15] > 1 ? S.hcnt[14] : 0;
        if (F.n_runs && (st = plan_runs_write(c, l + 1, cnt + 14))) return st;
        F.n_ghost = S.hcnt[4];
        if (F.n_ghost && (st = F.ghost.reserve((size_t)F.n_ghost * PSLOT))) return st;
        if (F.n_ghost && c->prm.scheme == AMR_SCHEME_VL && (st = F.ghost_ustar.reserve((size_t)F.n_ghost * PSLOT)))
            return st;
        if (F.n_ghost && c->prm.dual_energy && (st = F.ghost_S.reserve((size_t)F.n_ghost * PV))) return st;
        if ((st = cf_finish(c, l + 1, S.hcnt + 5))) return st;
        F.ghost_valid = false;
        if (G2) {
            G2->n_runs = S.hcnt[18] > 1 ? S.hcnt[17] : 0;
            if (G2->n_runs && (st = plan_runs_write(c, l + 2, cnt + 17))) return st;
            G2->n_ghost = S.hcnt[9];
            if (G2->n_ghost && (st = G2->ghost.reserve((size_t)G2->n_ghost * PSLOT))) return st;
            if (G2->n_ghost && c->prm.scheme == AMR_SCHEME_VL &&
                (st = G2->ghost_ustar.reserve((size_t)G2->n_ghost * PSLOT)))
                return st;
            if (G2->n_ghost && c->prm.dual_energy && (st = G2->ghost_S.reserve((size_t)G2->n_ghost * PV))) return st;
            if ((st = cf_finish(c, l + 2, S.hcnt + 10))) return st;
            G2->ghost_valid = false;
        }
    }
    if (c->prm.scheme == AMR_SCHEME_VL && nn && (st = F.ustar.reserve((size_t)nn * PSLOT))) return st;
    return AMR_OK;
}

// Host copies of a level's tables, refreshed after device-side regrids.
amr_status refresh_host_tables(amr_hydro_ctx *c, int level) {
    Level &L = c->lv[level];
    if (!L.host_stale) return AMR_OK;
    const size_t n = (size_t)L.n_patches;
    L.corner.resize(n * 3);
    L.sib.resize(n * 26);
    L.parent.assign(n, -1);
    L.child.assign(n, -1);
    amr_status st;
    if (n) {
        if ((st = cuda_fail(cudaMemcpyAsync(L.corner.data(), L.d_corner, 12 * n, cudaMemcpyDeviceToHost, c->stream),
                            "d2h")) ||
            (st = cuda_fail(cudaMemcpyAsync(L.sib.data(), L.d_sib, 104 * n, cudaMemcpyDeviceToHost, c->stream), "d2h")))
            return st;
        if (L.d_parent &&
            (st = cuda_fail(cudaMemcpyAsync(L.parent.data(), L.d_parent, 4 * n, cudaMemcpyDeviceToHost, c->stream),
                            "d2h")))
            return st;
        if (L.d_child &&
            (st = cuda_fail(cudaMemcpyAsync(L.child.data(), L.d_child, 4 * n, cudaMemcpyDeviceToHost, c->stream),
                            "d2h")))
            return st;
        if ((st = cuda_fail(cudaStreamSynchronize(c->stream), "sync"))) return st;
    }
    L.host_stale = false;
    return AMR_OK;
}

}  // namespace amrh

// Test hook (not part of the C ABI): whether level `level`'s z-runs (the
// device plan's, or single groups) equal what the host plan makes from the
// same neighbour table (chains, run length for the same grid and estimate,
// runs); *n_runs_out = the level's run count.  1: equal, 0: different,
// -1: a CUDA error.
extern "C" int amrh_selftest_level_runs(amr_hydro_ctx *c, int level, int *n_runs_out) {
    using namespace amrh;
    Level &L = c->lv[level];
    const int ng = L.n_groups;
    std::vector<int32_t> nbr((size_t)ng * 64);
    if (ng && cudaMemcpy(nbr.data(), L.nbr.p, 4 * nbr.size(), cudaMemcpyDeviceToHost) != cudaSuccess) return -1;
    std::vector<int32_t> chains, coff, runs, off;
    z_chains(ng, nbr.data(), chains, coff);
    const int len = choose_run_len(coff, c->n_sm * c->step_bps, c->prm.prec == AMR_FP64 ? 0.05 : 0.13);
    *n_runs_out = L.n_runs;
    if (len <= 1) return L.n_runs == 0 ? 1 : 0;
    cut_runs(chains, coff, len, runs, off);
    if (L.n_runs != (int)off.size() - 1) return 0;
    std::vector<int32_t> dr(runs.size()), doff(off.size());
    if (cudaMemcpy(dr.data(), L.runs.p, 4 * dr.size(), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(doff.data(), L.run_off.p, 4 * doff.size(), cudaMemcpyDeviceToHost) != cudaSuccess)
        return -1;
    // the same runs; closed cycles may come in another order than the host's
    // (which lists them after the open chains)
    std::vector<std::vector<int32_t>> a, b;
    for (size_t r = 0; r + 1 < off.size(); r++) {
        a.emplace_back(runs.begin() + off[r], runs.begin() + off[r + 1]);
        if (doff[r] < 0 || doff[r + 1] > (int)dr.size() || doff[r] > doff[r + 1]) return 0;
        b.emplace_back(dr.begin() + doff[r], dr.begin() + doff[r + 1]);
    }
    std::sort(a.begin(), a.end());
    std::sort(b.begin(), b.end());
    return a == b ? 1 : 0;
}
