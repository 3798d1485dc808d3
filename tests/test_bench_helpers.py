"""Host-side helpers of bench.py: the algorithmic flop count behind the roofline, the
time-to-energy rule, and the kernel-source digest that keeps a recorded ncu traffic
figure tied to the code it was measured on."""
import os
import shutil

import bench


def test_flops_per_quartet_hand_counts():
    # per primitive quartet: 2 sum_{n<=L} n_h(L-n) for the R recursion and
    # 2 min(A H1 H2 + A C H2, C H1 H2 + A C H1) for the contraction; 81 primitive
    # quartets (3 primitives per shell); 12 A C for the digestion
    # (ss|ss): L = 0: 2*1 + 2*(1 + 1) = 6
    assert bench.flops_per_quartet(0, 0) == 81 * 6 + 12
    # (pp|pp): n_h(4..0) = 35, 20, 10, 4, 1 -> 140; A = C = 9, H1 = H2 = 10:
    # 9*10*10 + 9*9*10 = 1710 -> 3420
    assert bench.flops_per_quartet(2, 2) == 81 * (140 + 3420) + 12 * 81
    # (dd|dd): n_h(8..0) = 165, 120, 84, 56, 35, 20, 10, 4, 1 -> 990; A = C = 36,
    # H1 = H2 = 35: 36*35*35 + 36*36*35 = 89460 -> 178920
    assert bench.flops_per_quartet(5, 5) == 81 * (990 + 178920) + 12 * 1296
    # (ps|ss): L = 1: 2*(4 + 1) = 10; A = 3, C = 1, H1 = 4, H2 = 1:
    # min(3*4*1 + 3*1*1, 1*4*1 + 3*1*4) = min(15, 16) = 15 -> 30
    assert bench.flops_per_quartet(1, 0) == 81 * (10 + 30) + 12 * 3


def test_time_to_energy_is_the_start_of_the_final_stay_within_tolerance():
    ref = -1.0
    res = {"energies": [-0.9, -1.0 + 5e-9, -1.0 + 2e-8, -1.0 + 3e-9, -1.0 - 1e-9],
           "times": [0.1, 0.2, 0.3, 0.4, 0.5]}
    assert bench.time_to_energy(res, ref) == 0.4  # the 5e-9 at 0.2 does not stay
    assert bench.time_to_energy({"energies": [-0.5, -0.9], "times": [0.1, 0.2]}, ref) is None


def test_kernel_digest_ignores_comments_but_not_code(tmp_path, monkeypatch):
    src = os.path.join(bench.ROOT, "paper_2510_24968_gb300", "csrc")
    dst = tmp_path / "paper_2510_24968_gb300" / "csrc"
    dst.mkdir(parents=True)
    for f in bench.KERNEL_SOURCES:
        shutil.copy(os.path.join(src, f), dst / f)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    d0 = bench.kernel_source_digest()
    f = dst / "eri_core.cuh"
    text = f.read_text()
    f.write_text("// an added comment line\n" + text.replace("namespace fsim {", "namespace fsim {  // note", 1))
    assert bench.kernel_source_digest() == d0
    f.write_text(text.replace("constexpr int kJKThreads = 128;", "constexpr int kJKThreads = 256;"))
    assert bench.kernel_source_digest() != d0


def test_pair_nnz_counts_the_non_vanishing_hermite_coefficients():
    # E^{ij}_t vanishes outside 0 <= t <= i + j (Sec. 2.1.3); for random exponents and
    # centres every coefficient inside that range is non-zero, so counting the oracle's
    # non-zero coefficients per component pair must give the closed product form
    from oracle import hermite_E
    for la, lb, ref in ((0, 0, 1), (1, 0, 6), (1, 1, 33), (2, 2, 336)):
        n = 0
        for ca in bench.cart_components(la):
            for cb in bench.cart_components(lb):
                cnt = 1
                for ax, X in enumerate((0.37, -0.52, 0.61)):
                    cnt *= sum(1 for t in range(la + lb + 1)
                               if abs(hermite_E(ca[ax], cb[ax], t, X, 0.8, 1.3)) > 1e-300)
                n += cnt
        assert n == ref == bench.pair_nnz(la, lb)


def test_method_flops_hand_counts():
    # (ss|ss): per primitive quartet R 2, ket transform 2*1*1, bra transform 2*1*1 / 9
    assert bench.method_flops_per_quartet(0, 0) == 81 * (2 + 2 + 2 / 9) + 12
    # (dd|dd): R 990, ket transform 2 * 35 * 336, bra transform 2 * 336 * 36 / 9
    assert bench.method_flops_per_quartet(5, 5) == 81 * (990 + 2 * 35 * 336 + 2 * 336 * 36 / 9) + 12 * 1296
    # never above the Hermite-dense count
    for X in range(6):
        for Y in range(X + 1):
            assert bench.method_flops_per_quartet(X, Y) <= bench.flops_per_quartet(X, Y)
