// Test harness (host only) for the multigrid setup code, which it links
// directly: reads a pencil from raw files, builds the hierarchy and writes
//   mg_host_dump <dir> layout <block> <R>: the finest level's fused-transfer
//       layouts (mg_fused_layout);
//   mg_host_dump <dir> eig <block> <level>: that level's dense pencil and its
//       eigendecomposition by mg_level_eig (V^T A V = diag(lam), V^T B V = I);
//   mg_host_dump <dir> nullspace <block> <n_null>: the hierarchy built from
//       the near-null space in <dir>/nul.bin (n x n_null float64; n_null = 0:
//       without one): level 0's P, rho and diagonal, level 1's pencil and
//       near-null space, every level's P (p<l>_*.bin) and the level sizes.
// <dir>/hdr.bin: int64 n, nnz; rp.bin, ci.bin (int32); a.bin, b.bin (float64).
#include <cstdio>
#include <string>
#include <vector>

#include "mg.h"

using namespace slrf;

template <class T> static bool rd(const std::string &f, std::vector<T> &v, size_t n) {
    v.resize(n);
    FILE *fp = fopen(f.c_str(), "rb");
    if (!fp) return false;
    const size_t r = fread(v.data(), sizeof(T), n, fp);
    fclose(fp);
    return r == n;
}
template <class T> static bool wr(const std::string &f, const std::vector<T> &v) {
    FILE *fp = fopen(f.c_str(), "wb");
    if (!fp) return false;
    const size_t r = fwrite(v.data(), sizeof(T), v.size(), fp);
    fclose(fp);
    return r == v.size();
}

int main(int argc, char **argv) {
    if (argc != 5) return 2;
    const std::string dir = argv[1], mode = argv[2];
    std::vector<long long> hdr;
    if (!rd(dir + "/hdr.bin", hdr, 2)) return 3;
    const int n = (int)hdr[0];
    const long long nnz = hdr[1];
    std::vector<int32_t> rp, ci;
    std::vector<double> a, b;
    if (!rd(dir + "/rp.bin", rp, n + 1) || !rd(dir + "/ci.bin", ci, nnz) || !rd(dir + "/a.bin", a, nnz) ||
        !rd(dir + "/b.bin", b, nnz))
        return 3;
    MgParams prm;
    prm.block = std::stoi(argv[3]);
    std::vector<double> nul;
    if (mode == "nullspace") {
        prm.n_null = std::stoi(argv[4]);
        if (prm.n_null > 0) {
            if (!rd(dir + "/nul.bin", nul, (size_t)n * prm.n_null)) return 3;
            prm.near_null = nul.data();
        }
    }
    HostHierarchy H;
    const std::string err = mg_build(n, rp.data(), ci.data(), a.data(), b.data(), prm, H);
    if (!err.empty() || H.lv.size() < 2) {
        fprintf(stderr, "%s\n", err.c_str());
        return 4;
    }
    if (mode == "eig") {
        const size_t l = (size_t)std::stoi(argv[4]);
        if (l < 1 || l >= H.lv.size()) return 2;
        const HostLevel &Lv = H.lv[l];
        const size_t m = (size_t)Lv.n;
        std::vector<double> Ad(m * m, 0.0), Bd(m * m, 0.0), V, lam;
        for (size_t i = 0; i < m; ++i)
            for (int32_t k = Lv.ptr[i]; k < Lv.ptr[i + 1]; ++k) {
                Ad[i * m + Lv.col[k]] = Lv.a[k];
                Bd[i * m + Lv.col[k]] = Lv.b[k];
            }
        const std::string e2 = mg_level_eig(Lv, V, lam);
        if (!e2.empty()) return 4;
        return wr(dir + "/Ad.bin", Ad) && wr(dir + "/Bd.bin", Bd) && wr(dir + "/V.bin", V) && wr(dir + "/lam.bin", lam)
                   ? 0
                   : 5;
    }
    if (mode == "nullspace") {
        const HostLevel &L0 = H.lv[0], &L1 = H.lv[1];
        std::vector<long long> sizes;
        for (const HostLevel &L : H.lv) sizes.push_back(L.n);
        const std::vector<double> r0 = {L0.rho};
        for (size_t l = 0; l + 1 < H.lv.size(); ++l) {   // every level's transfer
            const std::string s = dir + "/p" + std::to_string(l);
            if (!(wr(s + "_ptr.bin", H.lv[l].P.ptr) && wr(s + "_col.bin", H.lv[l].P.col) &&
                  wr(s + "_val.bin", H.lv[l].P.val)))
                return 5;
        }
        return wr(dir + "/sizes.bin", sizes) && wr(dir + "/p_ptr.bin", L0.P.ptr) && wr(dir + "/p_col.bin", L0.P.col) &&
                       wr(dir + "/p_val.bin", L0.P.val) && wr(dir + "/rho0.bin", r0) &&
                       wr(dir + "/diag0.bin", L0.diag_a) && wr(dir + "/l1_ptr.bin", L1.ptr) &&
                       wr(dir + "/l1_col.bin", L1.col) && wr(dir + "/l1_a.bin", L1.a) && wr(dir + "/l1_b.bin", L1.b) &&
                       wr(dir + "/l1_nul.bin", L1.nullspace)
                   ? 0
                   : 5;
    }
    if (mode != "layout") return 2;
    FusedLayout L;
    mg_fused_pattern(H.lv[0], H.lv[1].n, std::stoi(argv[4]), L);
    std::vector<double> q(L.q_count());
    mg_fused_values(H.lv[0], L, q.data());
    const std::vector<long long> out_hdr = {H.lv[1].n, (long long)L.up_col.size(), (long long)L.down_col.size()};
    return wr(dir + "/out_hdr.bin", out_hdr) && wr(dir + "/up_ptr.bin", L.up_ptr) && wr(dir + "/up_col.bin", L.up_col) &&
                   wr(dir + "/down_ptr.bin", L.down_ptr) && wr(dir + "/down_col.bin", L.down_col) &&
                   wr(dir + "/q.bin", q)
               ? 0
               : 5;
}
