/*
 * Oracle, block-structured refined grid (Sec. 4.1, 4.2.1).
 *
 * TEST INFRASTRUCTURE ONLY (see lbm_oracle.h).  Plain FP64 loops.
 *
 * Grid: levels l = 0..L-1 (L-1 finest), blocks of 16^3 cells, a level-(l+1)
 * cell is half the size of a level-l cell, 2:1 balance between neighbouring
 * blocks (Sec. 4.1).  Positions are in finest-level lattice units.
 *
 * Time stepping (Rohde's non-uniform scheme named in Sec. 4.1), read as:
 *   advance(l):
 *     explosion: every ghost cell of level l+1 takes the post-collision
 *       populations of the level-l cell containing it;
 *     advance(l+1) twice (finer levels take two steps per coarser step);
 *     update(l): each real level-l cell either pulls its populations from
 *       its neighbours (real or ghost cells of level l) or, if it is a host
 *       (a neighbour of the finer region), takes the average of its eight
 *       ghost sub-cells (coalescence); then collides.
 *       Active ghost cells of level l stream but do not collide.
 *
 * Non-equilibrium rescaling.  To first order in Chapman-Enskog a level-l
 * post-collision population carries f_neq = -(tau_l - 1) 3 w Q:grad u dx_l,
 * and one step of streaming over a distance d (in cells of that level)
 * adds -d 3 w Q:grad u dx.  In fine units a coarse post-collision value is
 * -(2 tau_c - 2) = -(tau_f - 3/2) (acoustic scaling: 2 tau_c = tau_f + 1/2).
 * The interface transfers above move populations between cell centres
 * that are 1.5 fine cells apart along the interface normal, so an exploded
 * value reaching the first fine cell arrives with -(tau_f - 3/2) - 3/2 =
 * -tau_f, the fine pre-collision value, and the coalesced mean of the
 * values streamed out of the fine region arrives at the host with
 * -(tau_f - 1) - 3/2 = -2 tau_c, the coarse pre-collision value.  The
 * transfers are therefore consistent without rescaling; rescaling them as
 * well would count the level change twice.  Populations that change level
 * in place, without streaming, are those of a regrid: a refined block's
 * cells take their parent's post-collision state and a coarsened cell the
 * mean of its eight children's.  Those are rescaled (rescale option) by
 * kappa = (tau_f - 1) / (2 (tau_c - 1)) per TRT part, or 1/kappa.
 *   On the finest level every step also runs the coupling of Algorithm 1.
 * Hosts are real level-l cells with a level-(l+1)-covered cell among their 26
 * neighbours; their sub-cells are the active ghost cells of level l+1.  Cells
 * at Chebyshev distance 2 from the finer region give static ghost cells
 * (they keep the exploded values while the active ones stream).
 *
 * Refinement (Sec. 4.2.1, Fig. "Refinement depending on the presence of a
 * particle"): the finest-level blocks that intersect the sphere's bounding
 * box (grown by one cell) and their 26 neighbours are finest; every coarser
 * level adds the 26 neighbours of the parents of the next finer level, which
 * keeps the 2:1 balance; blocks split into all eight children.
 */
#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <cstring>
#include <vector>

#include "common.h"
#include "lbm_oracle.h"

using namespace orc;

namespace {

constexpr int BS = 16;
constexpr int B3 = BS * BS * BS;

enum : int { LOC_NONE = 0, LOC_REAL = 1, LOC_GHOST = 2, LOC_WALL = 3 };

struct LevelData {
    int n[3] = {0, 0, 0};          // cells of the level across the domain
    int nb[3] = {0, 0, 0};         // block positions
    std::vector<int> map;          // block position -> real id (>= 0), ghost id (-2 - g), or -1
    std::vector<std::array<int, 3>> rpos, gpos;
    std::vector<double> rg, rg_new;   // real blocks, [block][q][cell]
    std::vector<double> gg, gg_new;   // ghost blocks
    std::vector<uint8_t> host;        // real cells: 1 host, 2 second ring, 0 otherwise
    std::vector<uint8_t> gkind;       // ghost cells: 1 active (host sub-cell), 2 static, 0 unused
    std::vector<uint8_t> flag;        // real cells of the finest level: 1 = inside the sphere
    double taup = 0, taum = 0, sp = 0, sm = 0, sb = 0;
};

}  // namespace

struct orc_amr {
    orc_amr_params p;
    int L = 1;
    std::vector<LevelData> lv;
    Particle part;
    double gravity[3] = {0, 0, 0};
    std::vector<double> history;
    std::atomic<int> error{0};          // 1: a pull found no source, 2: sphere left the finest level
    std::vector<int> substep;           // per level: index (0 or 1) of the current step within the coarser step
    bool have_box = false;
    double box_lo[3] = {0, 0, 0}, box_hi[3] = {0, 0, 0};
    double sensor_sigma = 0.0;          // flow sensor threshold sigma_c (0: off)
    double sensor_c = 0.0;              // coarsening factor c
};

namespace {

size_t pidx(int block, int q, int cell) { return ((size_t)block * 19 + q) * B3 + cell; }
int local_index(int x, int y, int z) { return (x % BS) + BS * ((y % BS) + BS * (z % BS)); }
int bpos_index(const LevelData& D, int bx, int by, int bz) { return bx + D.nb[0] * (by + D.nb[1] * bz); }

// Wraps or rejects global level coordinates.  false: outside through a wall.
bool wrap(const orc_amr* a, const LevelData& D, int c[3]) {
    for (int k = 0; k < 3; ++k) {
        if (c[k] < 0 || c[k] >= D.n[k]) {
            if (!a->p.periodic[k]) return false;
            c[k] = ((c[k] % D.n[k]) + D.n[k]) % D.n[k];
        }
    }
    return true;
}

// Finds the block holding global level cell c (already wrapped).
int locate(const LevelData& D, const int c[3], int* block, int* cell) {
    const int m = D.map[bpos_index(D, c[0] / BS, c[1] / BS, c[2] / BS)];
    *cell = local_index(c[0], c[1], c[2]);
    if (m >= 0) {
        *block = m;
        return LOC_REAL;
    }
    if (m <= -2) {
        *block = -2 - m;
        return LOC_GHOST;
    }
    return LOC_NONE;
}

// Relaxation times per level (acoustic scaling: dt and dx halve together, so
// tau - 1/2 halves from a level to the next coarser one; Lambda is the same
// on every level).
void level_rates(orc_amr* a) {
    for (int l = 0; l < a->L; ++l) {
        LevelData& D = a->lv[l];
        D.taup = 0.5 + (a->p.tau - 0.5) / (double)(1 << (a->L - 1 - l));
        D.taum = 0.5 + a->p.magic / (D.taup - 0.5);
        D.sp = 1.0 / D.taup;
        D.sm = 1.0 / D.taum;
        const double bulk = a->p.bulk > 0.0 ? a->p.bulk : 1.0;
        D.sb = bulk == 1.0 ? D.sp : 1.0 / (0.5 + bulk * (D.taup - 0.5));   // Lambda_b fixed on every level, like Lambda
    }
}

// Non-equilibrium rescaling factor between a coarse and the next finer level
// for post-collision populations: (tau_f - 1) / (2 (tau_c - 1)) for each of
// the symmetric (tau+) and antisymmetric (tau-) parts.
void kappa_c2f(const LevelData& C, const LevelData& F, double* kp, double* km) {
    *kp = std::fabs(C.taup - 1.0) < 1e-12 ? 1.0 : (F.taup - 1.0) / (2.0 * (C.taup - 1.0));
    *km = std::fabs(C.taum - 1.0) < 1e-12 ? 1.0 : (F.taum - 1.0) / (2.0 * (C.taum - 1.0));
}

// f = f_eq + kappa+ (f+ - f_eq+) + kappa- (f- - f_eq-), f_eq from the moments of f itself.
void rescale(double f[19], double kp, double km) {
    double drho = 0, u[3] = {0, 0, 0};
    for (int q = 0; q < 19; ++q) {
        drho += f[q];
        for (int k = 0; k < 3; ++k) u[k] += f[q] * C[q][k];
    }
    double out[19];
    const double e0 = geq(0, drho, u);
    out[0] = e0 + kp * (f[0] - e0);
    for (int q = 1; q < 19; q += 2) {
        const double eq = geq(q, drho, u), eb = geq(q + 1, drho, u);
        const double ep = 0.5 * (eq + eb), em = 0.5 * (eq - eb);
        const double fp = 0.5 * (f[q] + f[q + 1]), fm = 0.5 * (f[q] - f[q + 1]);
        out[q] = ep + kp * (fp - ep) + em + km * (fm - em);
        out[q + 1] = ep + kp * (fp - ep) - em - km * (fm - em);
    }
    std::memcpy(f, out, sizeof(out));
}

// Rescaling of post-collision states from level `from` to level `to` (one
// level at a time): refinement or coarsening of cells in a regrid.
void rescale_levels(const orc_amr* a, double f[19], int from, int to) {
    if (!a->p.rescale) return;
    while (from < to) {
        double kp, km;
        kappa_c2f(a->lv[from], a->lv[from + 1], &kp, &km);
        rescale(f, kp, km);
        ++from;
    }
    while (from > to) {
        double kp, km;
        kappa_c2f(a->lv[from - 1], a->lv[from], &kp, &km);
        rescale(f, kp != 0.0 ? 1.0 / kp : 1.0, km != 0.0 ? 1.0 / km : 1.0);
        --from;
    }
}

// TRT collision (Sec. 2.1) of one cell's deviations at level D; the MRT
// form when the bulk rate differs from s+ (Lambda_b != 1).
void collide(const LevelData& D, double g[19]) {
    double drho = 0, u[3] = {0, 0, 0};
    for (int q = 0; q < 19; ++q) {
        drho += g[q];
        for (int k = 0; k < 3; ++k) u[k] += g[q] * C[q][k];
    }
    if (D.sb != D.sp) {
        double ge[19], out[19];
        for (int q = 0; q < 19; ++q) ge[q] = geq(q, drho, u);
        mrt_collide(g, ge, nullptr, D.sp, D.sm, D.sb, out);
        std::memcpy(g, out, sizeof(out));
        return;
    }
    double out[19];
    const double e0 = geq(0, drho, u);
    out[0] = g[0] - D.sp * (g[0] - e0);
    for (int q = 1; q < 19; q += 2) {
        const double eq = geq(q, drho, u), eb = geq(q + 1, drho, u);
        const double gp = 0.5 * (g[q] + g[q + 1]), gm = 0.5 * (g[q] - g[q + 1]);
        const double ep = 0.5 * (eq + eb), em = 0.5 * (eq - eb);
        const double dp = D.sp * (gp - ep), dm = D.sm * (gm - em);
        out[q] = g[q] - dp - dm;
        out[q + 1] = g[q + 1] - dp + dm;
    }
    std::memcpy(g, out, sizeof(out));
}

// ----------------------------------------------------------- refinement
using Mask = std::vector<uint8_t>;

void level_lattice(const orc_amr* a, int l, int nb[3]) {
    const int n0[3] = {a->p.nx, a->p.ny, a->p.nz};
    for (int k = 0; k < 3; ++k) nb[k] = n0[k] * (1 << l) / BS;
}

Mask parents_of(const orc_amr* a, const Mask& fine, int lf) {
    int nbf[3], nbc[3];
    level_lattice(a, lf, nbf);
    level_lattice(a, lf - 1, nbc);
    Mask out((size_t)nbc[0] * nbc[1] * nbc[2], 0);
    for (int z = 0; z < nbf[2]; ++z)
        for (int y = 0; y < nbf[1]; ++y)
            for (int x = 0; x < nbf[0]; ++x)
                if (fine[x + nbf[0] * (y + nbf[1] * z)]) out[x / 2 + nbc[0] * (y / 2 + nbc[1] * (z / 2))] = 1;
    return out;
}

Mask children_of(const orc_amr* a, const Mask& coarse, int lc) {
    int nbf[3], nbc[3];
    level_lattice(a, lc + 1, nbf);
    level_lattice(a, lc, nbc);
    Mask out((size_t)nbf[0] * nbf[1] * nbf[2], 0);
    for (int z = 0; z < nbf[2]; ++z)
        for (int y = 0; y < nbf[1]; ++y)
            for (int x = 0; x < nbf[0]; ++x)
                out[x + nbf[0] * (y + nbf[1] * z)] = coarse[x / 2 + nbc[0] * (y / 2 + nbc[1] * (z / 2))];
    return out;
}

Mask grow26(const orc_amr* a, const Mask& m, int l) {
    int nb[3];
    level_lattice(a, l, nb);
    Mask out(m);
    for (int z = 0; z < nb[2]; ++z)
        for (int y = 0; y < nb[1]; ++y)
            for (int x = 0; x < nb[0]; ++x) {
                if (!m[x + nb[0] * (y + nb[1] * z)]) continue;
                for (int dz = -1; dz <= 1; ++dz)
                    for (int dy = -1; dy <= 1; ++dy)
                        for (int dx = -1; dx <= 1; ++dx) {
                            int c[3] = {x + dx, y + dy, z + dz};
                            bool ok = true;
                            for (int k = 0; k < 3; ++k) {
                                if (c[k] < 0 || c[k] >= nb[k]) {
                                    if (!a->p.periodic[k]) ok = false;
                                    else c[k] = (c[k] + nb[k]) % nb[k];
                                }
                            }
                            if (ok) out[c[0] + nb[0] * (c[1] + nb[1] * c[2])] = 1;
                        }
            }
    return out;
}

// R[l]: level-l block positions covered by blocks of level >= l.  demand[l]
// (optional, l >= 1) adds level-l positions that must be covered at level
// >= l (the flow sensor's wishes); the finest mask is demand[L-1]'s
// particle part.
std::vector<Mask> covered_sets(const orc_amr* a, const Mask& finest, const std::vector<Mask>* demand = nullptr) {
    const int L = a->L;
    std::vector<Mask> R(L);
    int nb[3];
    level_lattice(a, 0, nb);
    R[0].assign((size_t)nb[0] * nb[1] * nb[2], 1);
    if (L == 1) return R;
    Mask top = finest;
    if (demand)
        for (size_t i = 0; i < top.size(); ++i) top[i] |= (*demand)[L - 1][i];
    R[L - 1] = children_of(a, parents_of(a, top, L - 1), L - 2);   // all eight siblings
    for (int l = L - 2; l >= 1; --l) {
        Mask P = parents_of(a, R[l + 1], l + 1);
        Mask X = grow26(a, P, l);
        if (demand)
            for (size_t i = 0; i < X.size(); ++i) X[i] |= (*demand)[l][i];
        R[l] = children_of(a, parents_of(a, X, l), l - 1);
    }
    return R;
}

// Finest block positions intersecting the sphere's bounding box grown by one
// cell, plus their 26 neighbours.
Mask particle_mask(const orc_amr* a) {
    int nb[3];
    level_lattice(a, a->L - 1, nb);
    Mask m((size_t)nb[0] * nb[1] * nb[2], 0);
    int lo[3], hi[3];
    for (int k = 0; k < 3; ++k) {
        lo[k] = (int)std::floor((a->part.x[k] - a->part.r - 1.0) / BS);
        hi[k] = (int)std::floor((a->part.x[k] + a->part.r + 1.0) / BS);
    }
    for (int z = lo[2]; z <= hi[2]; ++z)
        for (int y = lo[1]; y <= hi[1]; ++y)
            for (int x = lo[0]; x <= hi[0]; ++x) {
                int c[3] = {x, y, z};
                bool ok = true;
                for (int k = 0; k < 3; ++k) {
                    if (c[k] < 0 || c[k] >= nb[k]) {
                        if (!a->p.periodic[k]) ok = false;
                        else c[k] = (c[k] % nb[k] + nb[k]) % nb[k];
                    }
                }
                if (ok) m[c[0] + nb[0] * (c[1] + nb[1] * c[2])] = 1;
            }
    return grow26(a, m, a->L - 1);
}

Mask box_mask(const orc_amr* a) {
    int nb[3];
    level_lattice(a, a->L - 1, nb);
    Mask m((size_t)nb[0] * nb[1] * nb[2], 0);
    for (int z = 0; z < nb[2]; ++z)
        for (int y = 0; y < nb[1]; ++y)
            for (int x = 0; x < nb[0]; ++x) {
                const int c[3] = {x, y, z};
                bool in = true;
                for (int k = 0; k < 3; ++k)
                    if (!((c[k] + 1) * BS > a->box_lo[k] && c[k] * BS < a->box_hi[k])) in = false;
                if (in) m[x + nb[0] * (y + nb[1] * z)] = 1;
            }
    return m;
}

// ------------------------------------------------------------- layout
// Builds the block sets of every level from the covered sets, the host and
// ghost classification, and moves the populations of the old layout over
// (copy, explosion from a coarser old cell, or coalescence of finer old cells).
void build_layout(orc_amr* a, const std::vector<Mask>& R) {
    const int L = a->L;
    std::vector<LevelData> old;
    old.swap(a->lv);
    a->lv.assign(L, LevelData());
    const int n0[3] = {a->p.nx, a->p.ny, a->p.nz};
    std::vector<Mask> refined(L);   // level-l positions whose children are covered
    for (int l = 0; l < L; ++l) {
        LevelData& D = a->lv[l];
        for (int k = 0; k < 3; ++k) {
            D.n[k] = n0[k] * (1 << l);
            D.nb[k] = D.n[k] / BS;
        }
        const size_t nbp = (size_t)D.nb[0] * D.nb[1] * D.nb[2];
        D.map.assign(nbp, -1);
        refined[l] = (l + 1 < L) ? parents_of(a, R[l + 1], l + 1) : Mask(nbp, 0);
        for (int z = 0; z < D.nb[2]; ++z)
            for (int y = 0; y < D.nb[1]; ++y)
                for (int x = 0; x < D.nb[0]; ++x) {
                    const int i = bpos_index(D, x, y, z);
                    if (R[l][i] && !refined[l][i]) {
                        D.map[i] = (int)D.rpos.size();
                        D.rpos.push_back({x, y, z});
                    }
                }
    }
    level_rates(a);
    // hosts and second-ring cells, ghost cells of the next level
    for (int l = 0; l + 1 < L; ++l) {
        LevelData& D = a->lv[l];
        LevelData& F = a->lv[l + 1];
        D.host.assign(D.rpos.size() * B3, 0);
        std::vector<std::array<int, 4>> subs;   // (x, y, z, kind) at level l+1
        for (size_t b = 0; b < D.rpos.size(); ++b)
            for (int c = 0; c < B3; ++c) {
                const int g[3] = {D.rpos[b][0] * BS + c % BS, D.rpos[b][1] * BS + (c / BS) % BS,
                                  D.rpos[b][2] * BS + c / (BS * BS)};
                int dist = 3;
                for (int dz = -2; dz <= 2; ++dz)
                    for (int dy = -2; dy <= 2; ++dy)
                        for (int dx = -2; dx <= 2; ++dx) {
                            int v[3] = {g[0] + dx, g[1] + dy, g[2] + dz};
                            if (!wrap(a, D, v)) continue;
                            if (refined[l][bpos_index(D, v[0] / BS, v[1] / BS, v[2] / BS)]) {
                                const int d = std::max(std::abs(dx), std::max(std::abs(dy), std::abs(dz)));
                                dist = std::min(dist, d);
                            }
                        }
                if (dist <= 2) {
                    const uint8_t kind = dist <= 1 ? 1 : 2;
                    D.host[b * B3 + c] = kind;
                    for (int s = 0; s < 8; ++s)
                        subs.push_back({2 * g[0] + (s & 1), 2 * g[1] + ((s >> 1) & 1), 2 * g[2] + (s >> 2), kind});
                }
            }
        // ghost blocks of level l+1 in position order
        Mask gmask((size_t)F.nb[0] * F.nb[1] * F.nb[2], 0);
        for (auto& s : subs) gmask[bpos_index(F, s[0] / BS, s[1] / BS, s[2] / BS)] = 1;
        for (int z = 0; z < F.nb[2]; ++z)
            for (int y = 0; y < F.nb[1]; ++y)
                for (int x = 0; x < F.nb[0]; ++x) {
                    const int i = bpos_index(F, x, y, z);
                    if (gmask[i]) {
                        F.map[i] = -2 - (int)F.gpos.size();
                        F.gpos.push_back({x, y, z});
                    }
                }
        F.gkind.assign(F.gpos.size() * B3, 0);
        for (auto& s : subs) {
            const int gid = -2 - F.map[bpos_index(F, s[0] / BS, s[1] / BS, s[2] / BS)];
            F.gkind[(size_t)gid * B3 + local_index(s[0], s[1], s[2])] = (uint8_t)s[3];
        }
    }
    // populations
    for (int l = 0; l < L; ++l) {
        LevelData& D = a->lv[l];
        D.rg.assign(D.rpos.size() * 19 * B3, 0.0);
        D.rg_new.assign(D.rpos.size() * 19 * B3, 0.0);
        D.gg.assign(D.gpos.size() * 19 * B3, 0.0);
        D.gg_new.assign(D.gpos.size() * 19 * B3, 0.0);
        D.flag.assign(D.rpos.size() * B3, 0);
        if (old.empty()) continue;
        for (size_t b = 0; b < D.rpos.size(); ++b)
            for (int c = 0; c < B3; ++c) {
                const int g[3] = {D.rpos[b][0] * BS + c % BS, D.rpos[b][1] * BS + (c / BS) % BS,
                                  D.rpos[b][2] * BS + c / (BS * BS)};
                double f[19] = {0};
                bool found = false;
                for (int lo = 0; lo < L && !found; ++lo) {
                    const LevelData& O = old[lo];
                    if (lo <= l) {   // old cell of level lo containing g
                        const int sh = l - lo;
                        const int v[3] = {g[0] >> sh, g[1] >> sh, g[2] >> sh};
                        int ob, oc;
                        if (locate(O, v, &ob, &oc) != LOC_REAL) continue;
                        for (int q = 0; q < 19; ++q) f[q] = O.rg[pidx(ob, q, oc)];
                        rescale_levels(a, f, lo, l);
                        found = true;
                    } else {         // average of the old finer cells inside g
                        const int k = 1 << (lo - l);
                        const int v0[3] = {g[0] * k, g[1] * k, g[2] * k};
                        int ob, oc;
                        if (locate(O, v0, &ob, &oc) != LOC_REAL) continue;
                        for (int dz = 0; dz < k; ++dz)
                            for (int dy = 0; dy < k; ++dy)
                                for (int dx = 0; dx < k; ++dx) {
                                    const int v[3] = {v0[0] + dx, v0[1] + dy, v0[2] + dz};
                                    locate(O, v, &ob, &oc);
                                    for (int q = 0; q < 19; ++q) f[q] += O.rg[pidx(ob, q, oc)];
                                }
                        for (int q = 0; q < 19; ++q) f[q] /= (double)(k * k * k);
                        rescale_levels(a, f, lo, l);
                        found = true;
                    }
                }
                for (int q = 0; q < 19; ++q) D.rg[pidx((int)b, q, c)] = f[q];
            }
    }
}

// --------------------------------------------------------------- sphere
bool inside(const orc_amr* a, const LevelData& D, const int g[3]) {
    const Particle& P = a->part;
    double d[3];
    for (int k = 0; k < 3; ++k) {
        d[k] = (g[k] + 0.5) - P.x[k];
        if (a->p.periodic[k]) {
            const double Lk = (double)D.n[k];
            if (d[k] > 0.5 * Lk) d[k] -= Lk;
            else if (d[k] < -0.5 * Lk) d[k] += Lk;
        }
    }
    return ((d[0] * d[0]) + (d[1] * d[1])) + (d[2] * d[2]) <= P.r * P.r;
}

void min_image(const orc_amr* a, const LevelData& D, const double x[3], double d[3]) {
    for (int k = 0; k < 3; ++k) {
        d[k] = x[k] - a->part.x[k];
        if (a->p.periodic[k]) {
            const double Lk = (double)D.n[k];
            if (d[k] > 0.5 * Lk) d[k] -= Lk;
            else if (d[k] < -0.5 * Lk) d[k] += Lk;
        }
    }
}

// Marks sphere cells on the finest level; errors if the sphere's bounding box
// (grown by 2) reaches a cell that is not a real finest cell.
void finest_flags(orc_amr* a, std::vector<uint8_t>& nf) {
    LevelData& D = a->lv[a->L - 1];
    nf.assign(D.rpos.size() * B3, 0);
    if (!a->part.present) return;
    for (size_t b = 0; b < D.rpos.size(); ++b)
        for (int c = 0; c < B3; ++c) {
            const int g[3] = {D.rpos[b][0] * BS + c % BS, D.rpos[b][1] * BS + (c / BS) % BS,
                              D.rpos[b][2] * BS + c / (BS * BS)};
            nf[b * B3 + c] = inside(a, D, g) ? 1 : 0;
        }
    const int R = (int)std::ceil(a->part.r) + 2;
    for (int dz = -R; dz <= R; ++dz)
        for (int dy = -R; dy <= R; ++dy)
            for (int dx = -R; dx <= R; ++dx) {
                int v[3] = {(int)std::floor(a->part.x[0]) + dx, (int)std::floor(a->part.x[1]) + dy,
                            (int)std::floor(a->part.x[2]) + dz};
                if (!wrap(a, D, v)) continue;
                int bb, cc;
                if (locate(D, v, &bb, &cc) != LOC_REAL) a->error = 2;
            }
}

// ---------------------------------------------------------- flow sensor
// Scaled curl of the velocity (Sec. 4.2.2, Eq. "sensor_curl"):
// phi_c = |curl u| s^((r+1)/r) with r = 2 and s the cell size; positions and
// derivatives are in finest-level units, so s = 2^(L-1-l) on level l.  The
// velocity of a cell is u = sum_q g_q c_q, the momentum of its stored
// (post-collision) deviations; a uniform body force shifts it by a constant,
// which the curl does not see.  Derivatives (the paper gives no stencil):
// central differences between the block's own cells, one-sided differences
// on the block's faces, so a block's value depends on its own cells only.
// A block's value is the largest phi_c of its cells.
double block_sensor(const orc_amr* a, int l, int b) {
    const LevelData& D = a->lv[l];
    const double s = (double)(1 << (a->L - 1 - l));
    std::vector<double> u((size_t)B3 * 3, 0.0);
    for (int c = 0; c < B3; ++c)
        for (int q = 0; q < 19; ++q)
            for (int k = 0; k < 3; ++k) u[(size_t)c * 3 + k] += D.rg[pidx(b, q, c)] * C[q][k];
    // d u_comp / d x_axis at local cell p
    auto deriv = [&](int comp, int axis, const int p[3]) {
        int lo[3] = {p[0], p[1], p[2]}, hi[3] = {p[0], p[1], p[2]};
        if (p[axis] > 0) lo[axis] -= 1;
        if (p[axis] < BS - 1) hi[axis] += 1;
        const double du = u[(size_t)local_index(hi[0], hi[1], hi[2]) * 3 + comp] -
                          u[(size_t)local_index(lo[0], lo[1], lo[2]) * 3 + comp];
        return du / ((double)(hi[axis] - lo[axis]) * s);
    };
    double phi = 0.0;
    for (int z = 0; z < BS; ++z)
        for (int y = 0; y < BS; ++y)
            for (int x = 0; x < BS; ++x) {
                const int p[3] = {x, y, z};
                const double wx = deriv(2, 1, p) - deriv(1, 2, p);
                const double wy = deriv(0, 2, p) - deriv(2, 0, p);
                const double wz = deriv(1, 0, p) - deriv(0, 1, p);
                const double curl = std::sqrt(wx * wx + wy * wy + wz * wz);
                phi = std::max(phi, curl * std::pow(s, 1.5));
            }
    return phi;
}

// Positions each level must keep covered because of the flow sensor
// (Sec. 4.2.2): a real block of level l asks for level l+1 (capped at the
// finest) when its value exceeds sigma_c, for level l-1 when it is below
// c sigma_c, else for its own level.  Asking for level t means the block's
// region is covered at level >= t: its children (t = l+1), itself (t = l)
// or its parent (t = l-1).  Coarsening then happens only where all eight
// siblings agree, one level per regrid.
std::vector<Mask> sensor_demands(const orc_amr* a) {
    const int L = a->L;
    std::vector<Mask> dm(L);
    for (int l = 0; l < L; ++l) {
        int nb[3];
        level_lattice(a, l, nb);
        dm[l].assign((size_t)nb[0] * nb[1] * nb[2], 0);
    }
    for (int l = 0; l < L; ++l) {
        const LevelData& D = a->lv[l];
        for (size_t b = 0; b < D.rpos.size(); ++b) {
            const double phi = block_sensor(a, l, (int)b);
            int t = l;
            if (phi > a->sensor_sigma) t = std::min(l + 1, L - 1);
            else if (phi < a->sensor_c * a->sensor_sigma) t = std::max(l - 1, 0);
            const int* p = D.rpos[b].data();
            if (t == l + 1) {
                int nf[3];
                level_lattice(a, t, nf);
                for (int s = 0; s < 8; ++s)
                    dm[t][(2 * p[0] + (s & 1)) + nf[0] * ((2 * p[1] + ((s >> 1) & 1)) + nf[1] * (2 * p[2] + (s >> 2)))] = 1;
            } else if (t == l) {
                dm[l][bpos_index(D, p[0], p[1], p[2])] = 1;
            } else {
                int nc[3];
                level_lattice(a, t, nc);
                dm[t][p[0] / 2 + nc[0] * (p[1] / 2 + nc[1] * (p[2] / 2))] = 1;
            }
        }
    }
    return dm;
}

// use_sensor: explicit regrids consult the flow sensor (when it is on);
// creation, a new sphere and a refined box do not.
void regrid_now(orc_amr* a, bool use_sensor = false) {
    Mask m;
    int nb[3];
    level_lattice(a, a->L - 1, nb);
    if (a->part.present) m = particle_mask(a);
    else if (a->have_box) m = box_mask(a);
    else m.assign((size_t)nb[0] * nb[1] * nb[2], 0);
    if (a->part.present && a->have_box) {
        Mask mb = box_mask(a);
        for (size_t i = 0; i < m.size(); ++i) m[i] |= mb[i];
    }
    if (use_sensor && a->sensor_sigma > 0.0) {
        const std::vector<Mask> dm = sensor_demands(a);
        build_layout(a, covered_sets(a, m, &dm));
    } else {
        build_layout(a, covered_sets(a, m));
    }
    LevelData& D = a->lv[a->L - 1];
    finest_flags(a, D.flag);
    for (size_t b = 0; b < D.rpos.size(); ++b)
        for (int c = 0; c < B3; ++c)
            if (D.flag[b * B3 + c])
                for (int q = 0; q < 19; ++q) D.rg[pidx((int)b, q, c)] = 0.0;
}

// ------------------------------------------------------------- stepping
void explode(orc_amr* a, int l) {
    LevelData& D = a->lv[l];
    LevelData& F = a->lv[l + 1];
    const long ngb = (long)F.gpos.size();
#pragma omp parallel for schedule(static)
    for (long gb = 0; gb < ngb; ++gb)
        for (int c = 0; c < B3; ++c) {
            if (!F.gkind[gb * B3 + c]) continue;
            const int g[3] = {F.gpos[gb][0] * BS + c % BS, F.gpos[gb][1] * BS + (c / BS) % BS,
                              F.gpos[gb][2] * BS + c / (BS * BS)};
            const int v[3] = {g[0] / 2, g[1] / 2, g[2] / 2};
            int pb, pc;
            if (locate(D, v, &pb, &pc) != LOC_REAL) {
                a->error = 1;
                continue;
            }
            for (int q = 0; q < 19; ++q) {
                F.gg[pidx((int)gb, q, c)] = D.rg[pidx(pb, q, pc)];
                F.gg_new[pidx((int)gb, q, c)] = D.rg[pidx(pb, q, pc)];
            }
        }
}

// Exploded value of population q at level-l+1 position p: the
// post-collision population of the level-l cell containing p.
double exploded(orc_amr* a, int l, const int p[3], int q) {
    const LevelData& D = a->lv[l];
    int v[3] = {p[0] >> 1, p[1] >> 1, p[2] >> 1};
    int b, c;
    if (!wrap(a, D, v) || locate(D, v, &b, &c) != LOC_REAL) {
        a->error = 1;
        return 0.0;
    }
    return D.rg[pidx(b, q, c)];
}

// Value of population q pulled into cell g (level l) from g - c_q: the
// post-collision value of a real cell, the current value of an active ghost
// cell, or bounce-back of the cell's own opposite population at a domain
// wall.  A static ghost stands for coarse content moving rigidly: at the
// s-th step of the current coarser step it supplies the exploded value of
// the coarser cell that contains (g - c_q) - s c_q.
double pull(orc_amr* a, int l, const int g[3], int q, bool self_real, int sb, int sc) {
    const LevelData& D = a->lv[l];
    int s[3] = {g[0] - C[q][0], g[1] - C[q][1], g[2] - C[q][2]};
    if (!wrap(a, D, s)) {
        const int o = opposite(q);
        return self_real ? D.rg[pidx(sb, o, sc)] : D.gg[pidx(sb, o, sc)];
    }
    int b, c;
    const int k = locate(D, s, &b, &c);
    if (k == LOC_REAL) return D.rg[pidx(b, q, c)];
    if (k == LOC_GHOST) {
        if (D.gkind[(size_t)b * B3 + c] == 1 || a->substep[l] == 0) return D.gg[pidx(b, q, c)];
        int t[3] = {s[0] - C[q][0], s[1] - C[q][1], s[2] - C[q][2]};
        if (!wrap(a, D, t)) return D.gg[pidx(b, q, c)];
        return exploded(a, l - 1, t, q);
    }
    a->error = 1;
    return 0.0;
}

// Finest-level CLI link (Sec. 2.3) for the cell at g pulling q from a solid
// cell; accumulates the link force and torque.
double cli_link(orc_amr* a, const LevelData& D, const int g[3], int qin, int sb, int sc, double F[3], double T[3]) {
    const Particle& P = a->part;
    const int q = opposite(qin);   // points from g into the solid
    double xc[3] = {g[0] + 0.5, g[1] + 0.5, g[2] + 0.5};
    double d[3];
    min_image(a, D, xc, d);
    double delta = 0.5;
    int far[3] = {g[0] - C[q][0], g[1] - C[q][1], g[2] - C[q][2]};
    int fb = -1, fc = -1;
    bool far_ok = wrap(a, D, far) && locate(D, far, &fb, &fc) == LOC_REAL && D.flag[(size_t)fb * B3 + fc] == 0;
    if (a->p.boundary == 0 && far_ok) {
        double cc = 0, dc = 0, dd = 0;
        for (int k = 0; k < 3; ++k) {
            cc += (double)(C[q][k] * C[q][k]);
            dc += d[k] * C[q][k];
            dd += d[k] * d[k];
        }
        double disc = dc * dc - cc * (dd - P.r * P.r);
        if (disc < 0) disc = 0;
        delta = std::min(1.0, std::max(0.0, (-dc - std::sqrt(disc)) / cc));
    }
    const double kappa0 = (1.0 - 2.0 * delta) / (1.0 + 2.0 * delta);
    const double alpha = 4.0 / (1.0 + 2.0 * delta);
    double arm[3], wr[3], vb[3];
    for (int k = 0; k < 3; ++k) arm[k] = d[k] + delta * C[q][k];
    cross(P.w, arm, wr);
    for (int k = 0; k < 3; ++k) vb[k] = P.u[k] + wr[k];
    const double vc = vb[0] * C[q][0] + vb[1] * C[q][1] + vb[2] * C[q][2];
    const double ft_q = W[q] + D.rg[pidx(sb, q, sc)];
    const double ft_qb = W[qin] + D.rg[pidx(sb, qin, sc)];
    const double ft_far = far_ok ? W[q] + D.rg[pidx(fb, q, fc)] : 0.0;
    const double fnew = ft_q + kappa0 * ft_far - kappa0 * ft_qb - alpha * (W[q] / CS2) * vc;
    double Fl[3], Tl[3];
    for (int k = 0; k < 3; ++k) Fl[k] = (C[q][k] - vb[k]) * ft_q - (C[qin][k] - vb[k]) * fnew;
    cross(arm, Fl, Tl);
    for (int k = 0; k < 3; ++k) {
        F[k] += Fl[k];
        T[k] += Tl[k];
    }
    return fnew - W[qin];
}

void update(orc_amr* a, int l, double F[3], double T[3]) {
    LevelData& D = a->lv[l];
    const bool finest = (l == a->L - 1);
    const bool coupled = finest && a->part.present;
    for (int k = 0; k < 3; ++k) F[k] = T[k] = 0.0;
    // blocks are independent (each writes its own cells); the link forces
    // and torques are summed per block in cell and q order and the block
    // sums in block order, so the result does not depend on the threads
    const long nrb = (long)D.rpos.size();
    std::vector<double> FT((size_t)nrb * 6, 0.0);
#pragma omp parallel for schedule(dynamic, 1)
    for (long b = 0; b < nrb; ++b)
        for (int c = 0; c < B3; ++c) {
            double* Fb = &FT[(size_t)b * 6];
            double* Tb = Fb + 3;
            const int g[3] = {D.rpos[b][0] * BS + c % BS, D.rpos[b][1] * BS + (c / BS) % BS,
                              D.rpos[b][2] * BS + c / (BS * BS)};
            double f[19];
            if (coupled && D.flag[b * B3 + c]) {
                for (int q = 0; q < 19; ++q) D.rg_new[pidx((int)b, q, c)] = 0.0;
                continue;
            }
            if (!finest && D.host[b * B3 + c] == 1) {
                // coalescence: mean of the eight ghost sub-cells after the two finer steps
                const LevelData& Fl = a->lv[l + 1];
                for (int q = 0; q < 19; ++q) f[q] = 0.0;
                for (int s = 0; s < 8; ++s) {
                    const int v[3] = {2 * g[0] + (s & 1), 2 * g[1] + ((s >> 1) & 1), 2 * g[2] + (s >> 2)};
                    int gb, gc;
                    if (locate(Fl, v, &gb, &gc) != LOC_GHOST) {
                        a->error = 1;
                        continue;
                    }
                    for (int q = 0; q < 19; ++q) f[q] += Fl.gg[pidx(gb, q, gc)];
                }
                for (int q = 0; q < 19; ++q) f[q] /= 8.0;
            } else {
                for (int q = 0; q < 19; ++q) {
                    if (coupled && q > 0) {
                        int s[3] = {g[0] - C[q][0], g[1] - C[q][1], g[2] - C[q][2]};
                        int sb, sc;
                        if (wrap(a, D, s) && locate(D, s, &sb, &sc) == LOC_REAL && D.flag[(size_t)sb * B3 + sc]) {
                            f[q] = cli_link(a, D, g, q, (int)b, c, Fb, Tb);
                            continue;
                        }
                    }
                    f[q] = pull(a, l, g, q, true, (int)b, c);
                }
            }
            collide(D, f);
            for (int q = 0; q < 19; ++q) D.rg_new[pidx((int)b, q, c)] = f[q];
        }
    for (long b = 0; b < nrb; ++b)
        for (int k = 0; k < 3; ++k) {
            F[k] += FT[(size_t)b * 6 + k];
            T[k] += FT[(size_t)b * 6 + 3 + k];
        }
    const long ngb = (long)D.gpos.size();
#pragma omp parallel for schedule(dynamic, 1)
    for (long b = 0; b < ngb; ++b)
        for (int c = 0; c < B3; ++c) {
            const uint8_t k = D.gkind[b * B3 + c];
            if (k == 0) continue;
            if (k == 2) {   // static ghost: keeps the exploded values
                for (int q = 0; q < 19; ++q) D.gg_new[pidx((int)b, q, c)] = D.gg[pidx((int)b, q, c)];
                continue;
            }
            const int g[3] = {D.gpos[b][0] * BS + c % BS, D.gpos[b][1] * BS + (c / BS) % BS,
                              D.gpos[b][2] * BS + c / (BS * BS)};
            for (int q = 0; q < 19; ++q) D.gg_new[pidx((int)b, q, c)] = pull(a, l, g, q, false, (int)b, c);
        }
    D.rg.swap(D.rg_new);
    D.gg.swap(D.gg_new);
}

// Remap on the finest level after the particle moved (Sec. 2.3 with the
// equilibrium refill of uncovered cells).
void remap(orc_amr* a) {
    LevelData& D = a->lv[a->L - 1];
    std::vector<uint8_t> nf;
    finest_flags(a, nf);
    const Particle& P = a->part;
    for (size_t b = 0; b < D.rpos.size(); ++b)
        for (int c = 0; c < B3; ++c) {
            const size_t x = b * B3 + c;
            const bool was = D.flag[x] == 0, is = nf[x] == 0;
            if (!was && is) {
                const int g[3] = {D.rpos[b][0] * BS + c % BS, D.rpos[b][1] * BS + (c / BS) % BS,
                                  D.rpos[b][2] * BS + c / (BS * BS)};
                double rsum = 0;
                int cnt = 0;
                for (int q = 1; q < 19; ++q) {
                    int v[3] = {g[0] + C[q][0], g[1] + C[q][1], g[2] + C[q][2]};
                    int nb_, nc_;
                    if (!wrap(a, D, v) || locate(D, v, &nb_, &nc_) != LOC_REAL) continue;
                    const size_t y = (size_t)nb_ * B3 + nc_;
                    if (D.flag[y] != 0 || nf[y] != 0) continue;
                    double r = 1.0;
                    for (int p = 0; p < 19; ++p) r += D.rg[pidx(nb_, p, nc_)];
                    rsum += r;
                    cnt += 1;
                }
                const double rho = cnt > 0 ? rsum / cnt : 1.0;
                const double xc[3] = {g[0] + 0.5, g[1] + 0.5, g[2] + 0.5};
                double d[3], wr[3];
                min_image(a, D, xc, d);
                cross(P.w, d, wr);
                const double u[3] = {P.u[0] + wr[0], P.u[1] + wr[1], P.u[2] + wr[2]};
                double S[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
                if (a->p.refill == 1) {   // face neighbours fluid before and after the move
                    double up[3][3], um[3][3];
                    bool okp[3], okm[3];
                    for (int ax = 0; ax < 3; ++ax)
                        for (int sgn = 0; sgn < 2; ++sgn) {
                            int v[3] = {g[0], g[1], g[2]};
                            v[ax] += sgn == 0 ? 1 : -1;
                            int nb_, nc_;
                            bool ok = wrap(a, D, v) && locate(D, v, &nb_, &nc_) == LOC_REAL;
                            if (ok) ok = D.flag[(size_t)nb_ * B3 + nc_] == 0 && nf[(size_t)nb_ * B3 + nc_] == 0;
                            double* uu = sgn == 0 ? up[ax] : um[ax];
                            uu[0] = uu[1] = uu[2] = 0.0;
                            if (ok)
                                for (int p = 0; p < 19; ++p)
                                    for (int k = 0; k < 3; ++k) uu[k] += D.rg[pidx(nb_, p, nc_)] * C[p][k];
                            (sgn == 0 ? okp : okm)[ax] = ok;
                        }
                    refill_strain(up, okp, um, okm, u, S);
                }
                for (int q = 0; q < 19; ++q)
                    D.rg[pidx((int)b, q, c)] = geq(q, rho - 1.0, u) + (a->p.refill == 1 ? grad_noneq(q, D.sp, S) : 0.0);
            } else if (was && !is) {
                for (int q = 0; q < 19; ++q) D.rg[pidx((int)b, q, c)] = 0.0;
            }
        }
    D.flag.swap(nf);
}

void advance(orc_amr* a, int l) {
    if (l + 1 < a->L) {
        explode(a, l);
        a->substep[l + 1] = 0;
        advance(a, l + 1);
        a->substep[l + 1] = 1;
        advance(a, l + 1);
    }
    double F[3], T[3];
    update(a, l, F, T);
    if (l == a->L - 1 && a->part.present) {
        const LevelData& D = a->lv[l];
        const double ext[3] = {(double)D.n[0], (double)D.n[1], (double)D.n[2]};
        particle_advance(a->part, F, T, a->gravity, a->p.force_average != 0, a->p.plain_mem != 0, a->p.periodic,
                         ext, a->history);
        remap(a);
    }
}

}  // namespace

extern "C" {

orc_amr* orc_amr_create(const orc_amr_params* p) {
    if (!p || p->levels < 1 || p->levels > 6 || p->tau <= 0.5) return nullptr;
    const int n0[3] = {p->nx, p->ny, p->nz};
    for (int k = 0; k < 3; ++k)
        if (n0[k] < BS || n0[k] % BS) return nullptr;
    orc_amr* a = new orc_amr();
    a->p = *p;
    a->L = p->levels;
    a->lv.clear();
    a->substep.assign(a->L, 0);
    regrid_now(a);
    return a;
}

void orc_amr_destroy(orc_amr* a) { delete a; }

int orc_amr_refine_box(orc_amr* a, const double lo[3], const double hi[3]) {
    a->have_box = true;
    for (int k = 0; k < 3; ++k) {
        a->box_lo[k] = lo[k];
        a->box_hi[k] = hi[k];
    }
    regrid_now(a);
    return a->error;
}

int orc_amr_add_sphere(orc_amr* a, const double pos[3], double diameter, double density_ratio, double cv,
                       double cv_omega, int fixed) {
    if (a->part.present || diameter <= 0 || density_ratio <= 0) return -1;
    Particle& P = a->part;
    P = Particle();
    P.present = true;
    if (fixed < 0 || fixed > 2) return -1;
    P.fixed = P.prev_fixed = fixed;
    for (int k = 0; k < 3; ++k) P.x[k] = pos[k];
    P.D = diameter;
    P.r = 0.5 * diameter;
    P.rho_p = density_ratio;
    P.cv = cv;
    P.cvw = cv_omega;
    P.V = M_PI * diameter * diameter * diameter / 6.0;
    regrid_now(a);
    return a->error;
}

void orc_amr_set_gravity(orc_amr* a, const double g[3]) {
    for (int k = 0; k < 3; ++k) a->gravity[k] = g[k];
}

void orc_amr_set_particle_velocity(orc_amr* a, const double u[3], const double w[3]) {
    for (int k = 0; k < 3; ++k) {
        a->part.u[k] = u[k];
        a->part.w[k] = w[k];
    }
}

int orc_amr_regrid(orc_amr* a) {
    regrid_now(a, true);
    return a->error;
}

int orc_amr_set_sensor(orc_amr* a, double sigma, double c) {
    if (sigma < 0.0 || (sigma > 0.0 && !(c > 0.0 && c < std::pow(2.0, -1.5)))) return -1;
    a->sensor_sigma = sigma;
    a->sensor_c = c;
    return 0;
}

int64_t orc_amr_block_sensor(const orc_amr* a, int level, double* out, int64_t cap) {
    if (level < 0 || level >= a->L) return -1;
    const LevelData& D = a->lv[level];
    const int64_t n = (int64_t)D.rpos.size();
    if (out)
        for (int64_t b = 0; b < n && b < cap; ++b) out[b] = block_sensor(a, level, (int)b);
    return n;
}

void orc_amr_init_linear(orc_amr* a, double rho, const double u0[3], const double A[9], const double x0[3]) {
    const int L = a->L;
    for (int l = 0; l < L; ++l) {
        LevelData& D = a->lv[l];
        const double h = (double)(1 << (L - 1 - l));
        for (size_t b = 0; b < D.rpos.size(); ++b)
            for (int c = 0; c < B3; ++c) {
                const int g[3] = {D.rpos[b][0] * BS + c % BS, D.rpos[b][1] * BS + (c / BS) % BS,
                                  D.rpos[b][2] * BS + c / (BS * BS)};
                double xr[3], uu[3];
                for (int k = 0; k < 3; ++k) xr[k] = (g[k] + 0.5) * h - x0[k];
                for (int i = 0; i < 3; ++i) uu[i] = u0[i] + A[3 * i] * xr[0] + A[3 * i + 1] * xr[1] + A[3 * i + 2] * xr[2];
                const bool solid = (l == L - 1) && D.flag[b * B3 + c];
                for (int q = 0; q < 19; ++q) D.rg[pidx((int)b, q, c)] = solid ? 0.0 : geq(q, rho - 1.0, uu);
            }
    }
}

void orc_amr_init_equilibrium(orc_amr* a, double rho, const double u[3], double amp, int dir, int axis) {
    const int L = a->L;
    for (int l = 0; l < L; ++l) {
        LevelData& D = a->lv[l];
        const double h = (double)(1 << (L - 1 - l));   // cell size in finest units
        const double Lax = (double)a->lv[L - 1].n[axis];
        for (size_t b = 0; b < D.rpos.size(); ++b)
            for (int c = 0; c < B3; ++c) {
                const int g[3] = {D.rpos[b][0] * BS + c % BS, D.rpos[b][1] * BS + (c / BS) % BS,
                                  D.rpos[b][2] * BS + c / (BS * BS)};
                double uu[3] = {u[0], u[1], u[2]};
                if (amp != 0.0) uu[dir] += amp * std::sin(2.0 * M_PI * (g[axis] + 0.5) * h / Lax);
                const bool solid = (l == L - 1) && D.flag[b * B3 + c];
                for (int q = 0; q < 19; ++q) D.rg[pidx((int)b, q, c)] = solid ? 0.0 : geq(q, rho - 1.0, uu);
            }
    }
}

int orc_amr_step(orc_amr* a, int n) {
    for (int i = 0; i < n && !a->error; ++i) advance(a, 0);
    return a->error;
}

int orc_amr_error(const orc_amr* a) { return a->error; }

void orc_amr_level_shape(const orc_amr* a, int level, int out[3]) {
    for (int k = 0; k < 3; ++k) out[k] = a->lv[level].n[k];
}

int64_t orc_amr_block_map(const orc_amr* a, int level, int32_t* out, int64_t cap) {
    const LevelData& D = a->lv[level];
    const int64_t n = (int64_t)D.map.size();
    if (out)
        for (int64_t i = 0; i < n && i < cap; ++i) out[i] = D.map[i] >= 0 ? D.map[i] : (D.map[i] <= -2 ? -2 : -1);
    return n;
}

void orc_amr_level_populations(const orc_amr* a, int level, double* out) {
    const LevelData& D = a->lv[level];
    const size_t n = (size_t)D.n[0] * D.n[1] * D.n[2];
    for (size_t i = 0; i < 19 * n; ++i) out[i] = NAN;
    for (size_t b = 0; b < D.rpos.size(); ++b)
        for (int c = 0; c < B3; ++c) {
            const size_t g = (size_t)(D.rpos[b][0] * BS + c % BS) +
                             (size_t)D.n[0] * ((size_t)(D.rpos[b][1] * BS + (c / BS) % BS) +
                                               (size_t)D.n[1] * (size_t)(D.rpos[b][2] * BS + c / (BS * BS)));
            for (int q = 0; q < 19; ++q) out[(size_t)q * n + g] = D.rg[pidx((int)b, q, c)];
        }
}

int64_t orc_amr_real_cells(const orc_amr* a, int level, int32_t* xyz, double* g, int64_t cap) {
    const LevelData& D = a->lv[level];
    int64_t m = 0;
    for (size_t b = 0; b < D.rpos.size(); ++b)
        for (int c = 0; c < B3; ++c, ++m) {
            if (m >= cap) continue;
            if (xyz) {
                xyz[3 * m] = D.rpos[b][0] * BS + c % BS;
                xyz[3 * m + 1] = D.rpos[b][1] * BS + (c / BS) % BS;
                xyz[3 * m + 2] = D.rpos[b][2] * BS + c / (BS * BS);
            }
            if (g)
                for (int q = 0; q < 19; ++q) g[19 * m + q] = D.rg[pidx((int)b, q, c)];
        }
    return (int64_t)D.rpos.size() * B3;
}

int64_t orc_amr_get_flags(const orc_amr* a, uint8_t* out, int64_t cap) {
    const LevelData& D = a->lv[a->L - 1];
    const int64_t n = (int64_t)D.rpos.size() * B3;
    if (!out || cap < n) return n;
    for (size_t b = 0; b < D.rpos.size(); ++b)
        for (int c = 0; c < B3; ++c) {
            const size_t x = b * B3 + c;
            if (D.flag[x]) {
                out[x] = 1;
                continue;
            }
            out[x] = 0;
            if (!a->part.present) continue;
            const int g[3] = {D.rpos[b][0] * BS + c % BS, D.rpos[b][1] * BS + (c / BS) % BS,
                              D.rpos[b][2] * BS + c / (BS * BS)};
            for (int q = 1; q < 19; ++q) {
                int v[3] = {g[0] + C[q][0], g[1] + C[q][1], g[2] + C[q][2]};
                int vb, vc;
                if (wrap(a, D, v) && locate(D, v, &vb, &vc) == LOC_REAL && D.flag[(size_t)vb * B3 + vc]) {
                    out[x] = 2;
                    break;
                }
            }
        }
    return n;
}

int64_t orc_amr_get_links(const orc_amr* a, int64_t* cell, int32_t* qout, double* delta, int64_t cap) {
    const LevelData& D = a->lv[a->L - 1];
    int64_t cnt = 0;
    if (!a->part.present) return 0;
    for (size_t b = 0; b < D.rpos.size(); ++b)
        for (int c = 0; c < B3; ++c) {
            if (D.flag[b * B3 + c]) continue;
            const int g[3] = {D.rpos[b][0] * BS + c % BS, D.rpos[b][1] * BS + (c / BS) % BS,
                              D.rpos[b][2] * BS + c / (BS * BS)};
            for (int q = 1; q < 19; ++q) {
                int v[3] = {g[0] + C[q][0], g[1] + C[q][1], g[2] + C[q][2]};
                int vb, vc;
                if (!wrap(a, D, v) || locate(D, v, &vb, &vc) != LOC_REAL || !D.flag[(size_t)vb * B3 + vc]) continue;
                if (cnt < cap) {
                    // smallest root s in [0, 1] of |x + s c_q - x_p| = r (Sec. 2.3), x the cell centre
                    const double xc[3] = {g[0] + 0.5, g[1] + 0.5, g[2] + 0.5};
                    double d[3];
                    min_image(a, D, xc, d);
                    double cc = 0, dc = 0, dd = 0;
                    for (int k = 0; k < 3; ++k) {
                        cc += (double)(C[q][k] * C[q][k]);
                        dc += d[k] * C[q][k];
                        dd += d[k] * d[k];
                    }
                    double disc = dc * dc - cc * (dd - a->part.r * a->part.r);
                    if (disc < 0) disc = 0;
                    cell[cnt] = (int64_t)g[0] + (int64_t)D.n[0] * ((int64_t)g[1] + (int64_t)D.n[1] * g[2]);
                    qout[cnt] = q;
                    delta[cnt] = std::min(1.0, std::max(0.0, (-dc - std::sqrt(disc)) / cc));
                }
                ++cnt;
            }
        }
    return cnt;
}

void orc_amr_mass(const orc_amr* a, double out[4]) {
    for (int k = 0; k < 4; ++k) out[k] = 0.0;
    for (int l = 0; l < a->L; ++l) {
        const LevelData& D = a->lv[l];
        const double vol = std::pow(8.0, a->L - 1 - l);
        for (size_t b = 0; b < D.rpos.size(); ++b)
            for (int c = 0; c < B3; ++c) {
                double r = 0, m[3] = {0, 0, 0};
                for (int q = 0; q < 19; ++q) {
                    const double v = D.rg[pidx((int)b, q, c)];
                    r += v;
                    for (int k = 0; k < 3; ++k) m[k] += v * C[q][k];
                }
                out[0] += r * vol;
                for (int k = 0; k < 3; ++k) out[1 + k] += m[k] * vol;
            }
    }
}

void orc_amr_get_particle(const orc_amr* a, double out[24]) {
    const Particle& P = a->part;
    for (int k = 0; k < 3; ++k) {
        out[k] = P.Fh[k];
        out[3 + k] = P.Th[k];
        out[6 + k] = P.x[k];
        out[9 + k] = P.u[k];
        out[12 + k] = P.w[k];
        out[15 + k] = P.a[k];
        out[18 + k] = P.b[k];
        out[21 + k] = P.Fp[k];
    }
}

int64_t orc_amr_get_history(const orc_amr* a, double* out, int64_t cap_steps) {
    const int64_t steps = (int64_t)(a->history.size() / 15);
    const int64_t m = steps < cap_steps ? steps : cap_steps;
    if (out && m > 0) std::memcpy(out, a->history.data(), sizeof(double) * 15 * (size_t)m);
    return steps;
}

}  // extern "C"
