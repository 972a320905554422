// Test harness (host only): builds the multigrid hierarchy of a pencil read
// from raw files and writes the finest level's fused-transfer layouts
// (mg_fused_layout) as raw files, for the CPU test that compares them with
// scipy products of the exported prolongator.
//   mg_layout_dump <dir> <block> <R>
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
    if (argc != 4) return 2;
    const std::string dir = argv[1];
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
    prm.block = std::stoi(argv[2]);
    HostHierarchy H;
    const std::string err = mg_build(n, rp.data(), ci.data(), a.data(), b.data(), prm, H);
    if (!err.empty() || H.lv.size() < 2) {
        fprintf(stderr, "%s\n", err.c_str());
        return 4;
    }
    FusedLayout L;
    mg_fused_layout(H.lv[0], H.lv[1].n, std::stoi(argv[3]), L);
    const std::vector<long long> out_hdr = {H.lv[1].n, (long long)L.up_col.size(), (long long)L.down_col.size()};
    return wr(dir + "/out_hdr.bin", out_hdr) && wr(dir + "/up_ptr.bin", L.up_ptr) && wr(dir + "/up_col.bin", L.up_col) &&
                   wr(dir + "/down_ptr.bin", L.down_ptr) && wr(dir + "/down_col.bin", L.down_col) &&
                   wr(dir + "/q.bin", L.q)
               ? 0
               : 5;
}
