"""Host logic of the benchmark: the algorithmic byte models behind its
roofline lines, summed from the records they name, and the DRAM traffic it
reports only while the committed ncu figure belongs to the current sweep
source."""
import hashlib
import os

import bench


def test_sweep_byte_models_are_the_records_they_name():
    # 2D FP64 contact: ids 8, normal 16, g/dt 8, m_n 8, m_t 8, impulse read 16 + write 16;
    # particle: (v, w) read + write 2 x 24, (inv_m, r, r/I) 24
    assert bench.sweep_bytes_model(2, "f64") == (8 + 16 + 8 + 8 + 8 + 16 + 16, 2 * 24 + 24)
    # FP32 halves the real-valued parts, not the ids
    assert bench.sweep_bytes_model(2, "f32") == (8 + (16 + 8 + 8 + 8 + 16 + 16) // 2, (2 * 24 + 24) // 2)
    # 3D FP64 contact: ids 8, geometry 32, (m_n, m_t) 16, impulse read 32 + write 32;
    # particle: v and w read + write 2 x 64, static 32
    assert bench.sweep_bytes_model(3, "f64") == (8 + 32 + 16 + 32 + 32, 2 * 64 + 32)


def test_detection_byte_model_is_the_records_it_names():
    for dim in (2, 3):
        pw = dim + 1 if dim == 3 else 2   # impulse components per contact
        contact = (8 + 24 + 8 + 8 + 8 + 8 * pw) + (8 + 8 * pw)   # record written, previous key + impulse read
        assert bench.detect_bytes_model(dim) == (contact, 8 * dim + 8)


def test_flops_per_update_are_the_listed_terms():
    # 2D: relative velocity, P_n, mu P_n, P_t, impulse change, its vector, both
    # bodies, |P| (4 + 1 for the square root)
    assert bench.FLOPS_PER_UPDATE_2D == (2 + 2 + 7) + 3 + 1 + 2 + 2 + 6 + 12 + (4 + 1)
    # 3D: lever sums, relative velocity, u_n, tangential part, P_n, trial P_t,
    # mu P_n, cone test, impulse change, its vector, n x dP, both bodies, |P|
    assert bench.FLOPS_PER_UPDATE_3D == 9 + 15 + 5 + 6 + 3 + 6 + 1 + 6 + 4 + 6 + 9 + 24 + 7


def _tree(root, src, line):
    os.makedirs(os.path.join(root, "paper_1104_3516_gb300", "csrc"))
    os.makedirs(os.path.join(root, "profiles"))
    with open(os.path.join(root, "paper_1104_3516_gb300", "csrc", "cd_sweep.cu"), "wb") as f:
        f.write(src)
    with open(os.path.join(root, "profiles", "k_sweep_traffic.txt"), "w") as f:
        f.write("# comment\n" + line + "\n")


def test_traffic_only_for_the_source_it_was_taken_with(tmp_path, monkeypatch):
    src = b"// a sweep kernel\n"
    sha = hashlib.sha256(src).hexdigest()[:16]
    line = (f"kernel=k_sweep<2,double> workload=w n=100000 precision=f64 traffic_bytes_per_launch=123 "
            f"src_sha256={sha}")
    _tree(str(tmp_path / "a"), src, line)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path / "a"))
    assert bench.profiled_traffic("k_sweep<2,double>", "f64", 100000) == 123.0
    assert bench.profiled_traffic("k_sweep<2,double>", "f64", 99999) is None
    assert bench.profiled_traffic("k_sweep<2,float>", "f32", 100000) is None
    # the kernel changed after the counters were taken: no figure
    _tree(str(tmp_path / "b"), src + b"// changed\n", line)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path / "b"))
    assert bench.profiled_traffic("k_sweep<2,double>", "f64", 100000) is None
