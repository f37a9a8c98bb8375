// Test driver: builds the library's host grid tables (grid.cpp, no GPU) and writes
// them as raw little-endian arrays so that the CPU tests can check them against
// the oracle.  Usage: host_grid_dump JMIN JMAX PATCH OUTDIR
#include <cstdio>
#include <cstdlib>
#include <string>
#include <vector>

#include "grid.h"

using namespace sww;

template <typename T>
static void put(const std::string& dir, const std::string& name, const std::vector<T>& v) {
    std::string path = dir + "/" + name;
    FILE* f = std::fopen(path.c_str(), "wb");
    if (!f) {
        std::perror(path.c_str());
        std::exit(2);
    }
    std::fwrite(v.data(), sizeof(T), v.size(), f);
    std::fclose(f);
}

template <typename T, int K>
static void put_slots(const std::string& dir, const std::string& name, const std::vector<T> (&v)[K], int n) {
    std::vector<T> flat;
    for (int k = 0; k < n; ++k) flat.insert(flat.end(), v[k].begin(), v[k].end());
    put(dir, name, flat);
}

int main(int argc, char** argv) {
    if (argc != 5) {
        std::fprintf(stderr, "usage: %s JMIN JMAX PATCH OUTDIR|--check|--check-corrupt\n", argv[0]);
        return 1;
    }
    int jmin = std::atoi(argv[1]), jmax = std::atoi(argv[2]), patch = std::atoi(argv[3]);
    std::string dir = argv[4];
    Hierarchy H;
    build_hierarchy(H, jmin, jmax, patch, 6.371e6, 7.292e-5);
    if (dir == "--check" || dir == "--check-corrupt") {
        // the table validator on the built grid, or on one planted out-of-range id
        if (dir == "--check-corrupt") H.lv[jmax].cor_i[3][H.lv[jmax].E / 2] = int32_t(H.lv[jmax].E);
        std::string what;
        const bool ok = validate_tables(H, &what);
        std::printf("%s\n", ok ? "tables ok" : what.c_str());
        return ok ? 0 : 3;
    }
    for (int j = jmin; j <= jmax; ++j) {
        HostLevel& L = H.lv[j];
        std::string p = "L" + std::to_string(j) + "_";
        std::vector<double> xyz;
        for (auto& x : L.xyz) xyz.push_back(x.x), xyz.push_back(x.y), xyz.push_back(x.z);
        put(dir, p + "xyz", xyz);
        put_slots(dir, p + "en", L.en, 2);
        put_slots(dir, p + "tn", L.tn, 3);
        put(dir, p + "A_i", L.A_i);
        put(dir, p + "A_v", L.A_v);
        put(dir, p + "d_e", L.d_e);
        put(dir, p + "l_e", L.l_e);
        put(dir, p + "f_v", L.f_v);
        put(dir, p + "f_n", L.f_n);
        put_slots(dir, p + "cor_i", L.cor_i, COR);
        put_slots(dir, p + "cor_w", L.cor_w, COR);
        put_slots(dir, p + "et", L.et, 2);
        put(dir, p + "tile_irr", L.tile_irr);
        put(dir, p + "tile_halo", L.tile_halo);
        if (j > jmin) {
            put_slots(dir, p + "par", L.par, 4);
            put_slots(dir, p + "akm", L.akm, 4);
            put_slots(dir, p + "ptw", L.ptw, 4);
            put_slots(dir, p + "vst", L.vst, VST);
            put_slots(dir, p + "vw", L.vw, VST);
        }
        if (j < jmax) {
            put(dir, p + "c2f", L.c2f);
            put_slots(dir, p + "half", L.half, 2);
            put_slots(dir, p + "mk_i", L.mk_i, 12);
            put_slots(dir, p + "mk_w", L.mk_w, 12);
            put_slots(dir, p + "rf_fi", L.rf_fi, RF_F);
            put_slots(dir, p + "rf_fw", L.rf_fw, RF_F);
            put_slots(dir, p + "rf_ci", L.rf_ci, RF_C);
            put_slots(dir, p + "rf_cw", L.rf_cw, RF_C);
        }
    }
    return 0;
}
