// mesh_host.cuh -- host-side mesh processing: faces and neighbours, periodic
// pairing, Morton locality order and per-cell geometry in the internal order.
#pragma once
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <map>
#include <string>
#include <unordered_map>
#include <vector>

#include "common.cuh"

namespace csw {

struct HostMesh {
    int nc = 0, ldc = 0;
    double rmin = 0.0;
    std::vector<int32_t> perm, iperm;     // internal -> user, user -> internal
    std::vector<double> vtx_user;         // 6 per user cell
    std::vector<double> geo, scv, arv;    // [G_COUNT][ldc]; sqrt(2/|K|); |K|
    std::vector<int32_t> nbr;             // [3][ldc]
    std::vector<uint8_t> nbfv;            // [ldc]
    std::vector<BFace> bfs;
    std::vector<double> vtx, nvtx;        // own vertices (6), neighbours' shifted vertices (3 x 6)
    std::string msg;
    int fail(int code, const char *fmt, ...)
    {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        msg = buf;
        return code;
    }
};

// Morton key of a point in the unit square (16 bits per axis)
inline uint32_t morton16(double x, double y)
{
    auto spread = [](uint32_t v) {
        v &= 0xffffu;
        v = (v | (v << 8)) & 0x00ff00ffu;
        v = (v | (v << 4)) & 0x0f0f0f0fu;
        v = (v | (v << 2)) & 0x33333333u;
        v = (v | (v << 1)) & 0x55555555u;
        return v;
    };
    const uint32_t ix = (uint32_t)std::min(65535.0, std::max(0.0, x * 65536.0));
    const uint32_t iy = (uint32_t)std::min(65535.0, std::max(0.0, y * 65536.0));
    return spread(ix) | (spread(iy) << 1);
}

// Returns 0 (CSWDG_OK) or a cswdg_status code with H.msg set.
inline int build_host_mesh(int k, const int32_t *bckind, int64_t nv, const double *xy, int64_t nc64, const int32_t *tri, int64_t nbf,
                           const int32_t *bface, const double *period, HostMesh &H)
{
    enum { EINVAL_ = 1, EMESH_ = 3 };
    const int BC_PER = 0;
    const int nc = (int)nc64;
    for (int64_t i = 0; i < 3 * nc64; ++i)
        if (tri[i] < 0 || tri[i] >= nv) return H.fail(EMESH_, "vertex index out of range");
    // ---- faces: pair half-edges by their sorted vertex pair ----
    struct HE { uint64_t key; int32_t cell; int32_t face; };
    std::vector<HE> he((size_t)3 * nc);
    for (int c = 0; c < nc; ++c)
        for (int f = 0; f < 3; ++f) {
            const uint64_t a = (uint64_t)tri[3 * c + f], b = (uint64_t)tri[3 * c + (f + 1) % 3];
            he[(size_t)3 * c + f] = HE{std::min(a, b) * (uint64_t)nv + std::max(a, b), c, f};
        }
    std::sort(he.begin(), he.end(), [](const HE &x, const HE &y) { return x.key < y.key || (x.key == y.key && x.cell < y.cell); });
    std::vector<int32_t> nb((size_t)3 * nc, -1), nbfl((size_t)3 * nc, -1), btag((size_t)3 * nc, -1);
    std::vector<double> shx((size_t)3 * nc, 0.0), shy((size_t)3 * nc, 0.0);
    for (size_t i = 0; i < he.size();) {
        size_t j = i + 1;
        while (j < he.size() && he[j].key == he[i].key) ++j;
        if (j - i == 2) {
            nb[3 * he[i].cell + he[i].face] = he[i + 1].cell;
            nbfl[3 * he[i].cell + he[i].face] = he[i + 1].face;
            nb[3 * he[i + 1].cell + he[i + 1].face] = he[i].cell;
            nbfl[3 * he[i + 1].cell + he[i + 1].face] = he[i].face;
        } else if (j - i > 2) {
            return H.fail(EMESH_, "edge shared by more than two triangles");
        }
        i = j;
    }
    std::unordered_map<uint64_t, int32_t> tagmap;
    for (int64_t e = 0; e < nbf; ++e) {
        const uint64_t a = (uint64_t)bface[3 * e], b = (uint64_t)bface[3 * e + 1];
        tagmap[std::min(a, b) * (uint64_t)nv + std::max(a, b)] = bface[3 * e + 2];
    }
    std::vector<int> per;
    for (int c = 0; c < nc; ++c)
        for (int f = 0; f < 3; ++f) {
            if (nb[3 * c + f] >= 0) continue;
            const uint64_t a = (uint64_t)tri[3 * c + f], b = (uint64_t)tri[3 * c + (f + 1) % 3];
            auto it = tagmap.find(std::min(a, b) * (uint64_t)nv + std::max(a, b));
            if (it == tagmap.end()) return H.fail(EMESH_, "boundary edge of cell %d has no tag", c);
            const int tag = it->second;
            if (tag < 0 || tag >= CSW_MAXTAG || bckind[tag] < 0) return H.fail(EMESH_, "boundary tag %d has no kind", tag);
            btag[3 * c + f] = tag;
            if (bckind[tag] == BC_PER) per.push_back(3 * c + f);
        }
    // ---- periodic pairing by translation of the edge midpoints ----
    if (!per.empty()) {
        if (!period) return H.fail(EINVAL_, "periodic faces but no period");
        const double Lx = period[0], Ly = period[1];
        const double q = 1e-7 * (std::fabs(Lx) + std::fabs(Ly));
        auto mid = [&](int hf, double &mx, double &my) {
            const int c = hf / 3, f = hf % 3;
            mx = 0.5 * (xy[2 * tri[3 * c + f]] + xy[2 * tri[3 * c + (f + 1) % 3]]);
            my = 0.5 * (xy[2 * tri[3 * c + f] + 1] + xy[2 * tri[3 * c + (f + 1) % 3] + 1]);
        };
        std::map<std::pair<long long, long long>, int> where;
        for (int hf : per) {
            double mx, my;
            mid(hf, mx, my);
            where[{llround(mx / q), llround(my / q)}] = hf;
        }
        for (int hf : per) {
            if (nb[hf] >= 0) continue;
            double mx, my;
            mid(hf, mx, my);
            const double cand[4][2] = {{Lx, 0.0}, {-Lx, 0.0}, {0.0, Ly}, {0.0, -Ly}};
            int partner = -1;
            double sx = 0.0, sy = 0.0;
            for (int k = 0; k < 4 && partner < 0; ++k) {
                auto it = where.find({llround((mx + cand[k][0]) / q), llround((my + cand[k][1]) / q)});
                if (it != where.end() && it->second != hf && nb[it->second] < 0) {
                    partner = it->second;
                    sx = -cand[k][0];
                    sy = -cand[k][1];
                }
            }
            if (partner < 0) return H.fail(EMESH_, "unpaired periodic face of cell %d", hf / 3);
            nb[hf] = partner / 3; nbfl[hf] = partner % 3; shx[hf] = sx; shy[hf] = sy;
            nb[partner] = hf / 3; nbfl[partner] = hf % 3; shx[partner] = -sx; shy[partner] = -sy;
        }
    }
    // ---- Morton locality order of the centroids ----
    double xmin = 1e300, xmax = -1e300, ymin = 1e300, ymax = -1e300;
    for (int64_t i = 0; i < nv; ++i) {
        xmin = std::min(xmin, xy[2 * i]); xmax = std::max(xmax, xy[2 * i]);
        ymin = std::min(ymin, xy[2 * i + 1]); ymax = std::max(ymax, xy[2 * i + 1]);
    }
    const double ext = std::max(xmax - xmin, ymax - ymin) * (1.0 + 1e-9) + 1e-300;
    std::vector<std::pair<uint32_t, int32_t>> key((size_t)nc);
    for (int c = 0; c < nc; ++c) {
        double cx = 0.0, cy = 0.0;
        for (int i = 0; i < 3; ++i) { cx += xy[2 * tri[3 * c + i]]; cy += xy[2 * tri[3 * c + i] + 1]; }
        key[c] = {morton16((cx / 3.0 - xmin) / ext, (cy / 3.0 - ymin) / ext), c};
    }
    std::sort(key.begin(), key.end());
    H.nc = nc;
    H.ldc = (nc + 31) & ~31;
    H.perm.assign(nc, 0);
    H.iperm.assign(nc, 0);
    for (int i = 0; i < nc; ++i) { H.perm[i] = key[i].second; H.iperm[key[i].second] = i; }
    H.vtx_user.assign((size_t)6 * nc, 0.0);
    for (int c = 0; c < nc; ++c)
        for (int i = 0; i < 3; ++i) {
            H.vtx_user[6 * c + 2 * i] = xy[2 * tri[3 * c + i]];
            H.vtx_user[6 * c + 2 * i + 1] = xy[2 * tri[3 * c + i] + 1];
        }
    // ---- geometry in internal order ----
    const int ld = H.ldc;
    std::vector<double> &geo = H.geo, &scv = H.scv, &arv = H.arv;
    geo.assign((size_t)G_COUNT * ld, 0.0); scv.assign(ld, 0.0); arv.assign(ld, 0.0);
    std::vector<int32_t> &nbr = H.nbr;
    nbr.assign((size_t)3 * ld, 0);
    std::vector<uint8_t> &nbfv = H.nbfv;
    nbfv.assign(ld, 0);
    std::vector<BFace> &bfs = H.bfs;
    bfs.clear();
    std::vector<double> &vtx = H.vtx, &nvtx = H.nvtx;
    vtx.assign((size_t)6 * nc, 0.0); nvtx.assign((size_t)18 * nc, 0.0);
    double rmin = 1e300;
    for (int i = 0; i < nc; ++i) {
        const int c = H.perm[i];
        double X[3], Y[3];
        for (int v = 0; v < 3; ++v) { X[v] = xy[2 * tri[3 * c + v]]; Y[v] = xy[2 * tri[3 * c + v] + 1]; }
        for (int v = 0; v < 3; ++v) { vtx[6 * i + 2 * v] = X[v]; vtx[6 * i + 2 * v + 1] = Y[v]; }
        const double a11 = X[1] - X[0], a12 = X[2] - X[0], a21 = Y[1] - Y[0], a22 = Y[2] - Y[0];
        const double det = a11 * a22 - a12 * a21, K = 0.5 * det;
        if (!(K > 0.0)) return H.fail(EMESH_, "triangle %d is not counter-clockwise or degenerate", c);
        geo[G_RX * ld + i] = 4.0 * a22 / det;
        geo[G_RY * ld + i] = -4.0 * a12 / det;
        geo[G_SX * ld + i] = -4.0 * a21 / det;
        geo[G_SY * ld + i] = 4.0 * a11 / det;
        double len[3], per_ = 0.0;
        for (int f = 0; f < 3; ++f) {
            const double dx = X[(f + 1) % 3] - X[f], dy = Y[(f + 1) % 3] - Y[f];
            len[f] = std::sqrt(dx * dx + dy * dy);
            per_ += len[f];
            geo[(G_N0X + 3 * f) * ld + i] = dy / len[f];
            geo[(G_N0Y + 3 * f) * ld + i] = -dx / len[f];
            geo[(G_N0L + 3 * f) * ld + i] = 2.0 * len[f] / K;
        }
        const double hc = len[0] * len[1] * len[2] / (4.0 * K);
        // KXRCF denominator factor h^{(k+1)/2} ||.||: the cell's L2 norm over its normalised
        // measure is sqrt(sum u~_m^2 / 2) for the stored coefficients u~ = sqrt(2/|K|) u^
        geo[G_KAPPA * ld + i] = ((k == 1) ? hc : hc * std::sqrt(hc)) * std::sqrt(0.5);
        scv[i] = std::sqrt(2.0 / K);
        arv[i] = K;
        rmin = std::min(rmin, 2.0 * K / per_);
        uint8_t bits = 0;
        for (int f = 0; f < 3; ++f) {
            const int h = 3 * c + f;
            if (nb[h] >= 0) {
                nbr[f * ld + i] = H.iperm[nb[h]];
                bits |= (uint8_t)(nbfl[h] << (2 * f));
                const int d = nb[h];
                for (int v = 0; v < 3; ++v) {
                    nvtx[(3 * (size_t)i + f) * 6 + 2 * v] = xy[2 * tri[3 * d + v]] + shx[h];
                    nvtx[(3 * (size_t)i + f) * 6 + 2 * v + 1] = xy[2 * tri[3 * d + v] + 1] + shy[h];
                }
            } else {
                BFace b{};
                b.ax = X[f]; b.ay = Y[f]; b.bx = X[(f + 1) % 3]; b.by = Y[(f + 1) % 3];
                b.nx = (b.by - b.ay) / len[f];
                b.ny = -(b.bx - b.ax) / len[f];
                b.tag = btag[h];
                nbr[f * ld + i] = -(int32_t)bfs.size() - 1;
                bfs.push_back(b);
            }
        }
        nbfv[i] = bits;
    }
    H.rmin = rmin;
    
    return 0;
}

}  // namespace csw
