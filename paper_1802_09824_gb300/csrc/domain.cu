// Domain decomposition for several GPUs (Sec. 4.1), host side.
//
// The box is cut along the space-filling curve of its ground cells (the
// cells of side >= rcut that the tree build starts from): every domain is a
// run of consecutive cells on the curve, runs chosen so that the domains
// carry about the same work.  The work of a cell is its particle count
// times the particle count of its 27-cell neighbourhood (the pairs its
// particles can reach within rcut).  A domain's ghost layer is the cells in
// the periodic 26-neighbourhood of its own cells that it does not own:
// since cells are at least rcut wide, its own cells plus the ghost cells
// hold every particle within rcut of any particle it owns (the argument of
// Sec. 4.3 for the 27-cell task), so a domain computes its particles'
// short-range forces from its local set alone.  Everything here runs on the
// host and needs no GPU.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "curve.cuh"
#include "phpp_internal.cuh"

using namespace phpp;

namespace {

// Ground cell coordinate of a wrapped coordinate: floor(2^g (x / L)) with
// x / L taken as x * fl(1 / L), clamped to the grid; the tree build's keys
// give the same cell (they quantise x * 2^T fl(1 / L) and drop T - g bits).
int cell_coord(double xw, double invL, int g)
{
    const double u = std::ldexp(xw * invL, g);
    const int nside = 1 << g;
    int c = (int)std::floor(u);
    return c < 0 ? 0 : (c >= nside ? nside - 1 : c);
}

double wrap64(double x, double L)
{
    if (x >= 0.0 && x < L) return x;
    return x - L * std::floor(x / L);
}

bool valid_nside(int32_t nside, int &g)
{
    for (g = 0; g <= kGroundMax; g++)
        if ((1 << g) == nside) return true;
    return false;
}

}  // namespace

extern "C" {

int ph_domain_cells(const void *pos, int pos_type, int64_t n, const ph_params *params, int32_t *nside, int32_t *cell)
{
    if (!params || !nside || (n > 0 && (!pos || !cell))) return fail(PH_ERR_ARG, "NULL argument");
    if (pos_type != PH_F32 && pos_type != PH_F64) return fail(PH_ERR_ARG, "pos_type must be PH_F32 or PH_F64");
    if (n < 0) return fail(PH_ERR_ARG, "n must be >= 0");
    const double L = params->L, rcut = params->rcut;
    if (!(std::isfinite(L) && L > 0 && std::isfinite(rcut) && rcut > 0 && rcut < 0.5 * L))
        return fail(PH_ERR_ARG, "need 0 < rcut < L/2");
    const int g = ground_level(L, rcut);
    const double invL = 1.0 / L;
    const float L_up = float_at_or_above(L);
    *nside = 1 << g;
    for (int64_t i = 0; i < n; i++) {
        int c[3];
        for (int a = 0; a < 3; a++) {
            double xw;
            if (pos_type == PH_F32) {
                const float x = static_cast<const float *>(pos)[3 * i + a];
                if (!std::isfinite(x)) return fail(PH_ERR_NONFINITE, "non-finite position at row %lld", (long long)i);
                xw = (x >= 0.f && x < L_up) ? (double)x : wrap64((double)x, L);
            } else {
                const double x = static_cast<const double *>(pos)[3 * i + a];
                if (!std::isfinite(x)) return fail(PH_ERR_NONFINITE, "non-finite position at row %lld", (long long)i);
                xw = wrap64(x, L);
            }
            c[a] = cell_coord(xw, invL, g);
        }
        cell[i] = (c[0] * *nside + c[1]) * *nside + c[2];
    }
    return PH_OK;
}

int ph_domain_partition(const int64_t *cell_count, int32_t nside, int32_t key_kind, int32_t n_domains, int32_t *owner,
                        double *domain_cost)
{
    int g = 0;
    if (!cell_count || !owner) return fail(PH_ERR_ARG, "NULL argument");
    if (!valid_nside(nside, g)) return fail(PH_ERR_ARG, "nside must be a power of two up to %d", 1 << kGroundMax);
    if (n_domains < 1) return fail(PH_ERR_ARG, "n_domains must be >= 1");
    if (key_kind != PH_KEY_MORTON && key_kind != PH_KEY_HILBERT) return fail(PH_ERR_ARG, "unknown key_kind");
    const int64_t cells = (int64_t)nside * nside * nside;
    std::vector<double> cost(cells);
    for (int i = 0; i < nside; i++)
        for (int j = 0; j < nside; j++)
            for (int k = 0; k < nside; k++) {
                double reach = 0.0;
                for (int di = -1; di <= 1; di++)
                    for (int dj = -1; dj <= 1; dj++)
                        for (int dk = -1; dk <= 1; dk++) {
                            const int a = (i + di + nside) % nside, b = (j + dj + nside) % nside,
                                      c = (k + dk + nside) % nside;
                            reach += (double)cell_count[((int64_t)a * nside + b) * nside + c];
                        }
                const int64_t id = ((int64_t)i * nside + j) * nside + k;
                if (cell_count[id] < 0) return fail(PH_ERR_ARG, "negative cell count");
                cost[id] = (double)cell_count[id] * reach;
            }
    // cells in curve order
    std::vector<uint64_t> key(cells);
    for (int64_t id = 0; id < cells; id++) {
        const uint32_t i = (uint32_t)(id / ((int64_t)nside * nside)), j = (uint32_t)((id / nside) % nside),
                       k = (uint32_t)(id % nside);
        key[id] = key_kind == PH_KEY_HILBERT ? hilbert3(i, j, k, g) : interleave3(i, j, k);
    }
    std::vector<int64_t> order(cells);
    std::iota(order.begin(), order.end(), 0);
    std::sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return key[a] < key[b]; });
    double total = 0.0;
    for (double c : cost) total += c;
    // a cell goes to the domain holding the midpoint of its cost on the
    // cumulative scale (cells of no cost: by position on the curve)
    double before = 0.0;
    for (int64_t p = 0; p < cells; p++) {
        const int64_t id = order[p];
        const double mid = total > 0 ? (before + 0.5 * cost[id]) / total : (p + 0.5) / (double)cells;
        int d = (int)std::floor(mid * n_domains);
        owner[id] = d < 0 ? 0 : (d >= n_domains ? n_domains - 1 : d);
        before += cost[id];
    }
    if (domain_cost) {
        for (int d = 0; d < n_domains; d++) domain_cost[d] = 0.0;
        for (int64_t id = 0; id < cells; id++) domain_cost[owner[id]] += cost[id];
    }
    return PH_OK;
}

int ph_domain_halo(const int32_t *owner, int32_t nside, int32_t domain, uint8_t *need)
{
    int g = 0;
    if (!owner || !need) return fail(PH_ERR_ARG, "NULL argument");
    if (!valid_nside(nside, g)) return fail(PH_ERR_ARG, "nside must be a power of two up to %d", 1 << kGroundMax);
    const int64_t cells = (int64_t)nside * nside * nside;
    for (int64_t id = 0; id < cells; id++) need[id] = owner[id] == domain ? 1 : 0;
    for (int i = 0; i < nside; i++)
        for (int j = 0; j < nside; j++)
            for (int k = 0; k < nside; k++) {
                if (owner[((int64_t)i * nside + j) * nside + k] != domain) continue;
                for (int di = -1; di <= 1; di++)
                    for (int dj = -1; dj <= 1; dj++)
                        for (int dk = -1; dk <= 1; dk++) {
                            const int a = (i + di + nside) % nside, b = (j + dj + nside) % nside,
                                      c = (k + dk + nside) % nside;
                            uint8_t &v = need[((int64_t)a * nside + b) * nside + c];
                            if (v == 0) v = 2;
                        }
            }
    return PH_OK;
}

}  // extern "C"
