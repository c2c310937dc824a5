"""Host-side checks of the build helpers: the kernel source hash that keys the
stored ncu traffic ignores comments and whitespace but not code."""
from paper_1304_7054_gb300 import build as lb


def test_strip_comments_keeps_literals_and_code():
    src = 'int a = 1; // note\n/* block\n */ const char* s = "x // y /* z */"; char q = \'"\'; b = a / 2;'
    out = lb.strip_comments(src)
    assert "note" not in out and "block" not in out
    assert '"x // y /* z */"' in out and "'\"'" in out and "b = a / 2;" in out


def test_hash_ignores_comments_and_whitespace_only(tmp_path, monkeypatch):
    d = tmp_path / "csrc"
    d.mkdir()
    f = d / "k.cu"
    monkeypatch.setattr(lb, "CSRC", str(d))
    monkeypatch.setitem(lb.FAMILY_SOURCES, "probe_kernel", ["k.cu"])
    f.write_text("__global__ void k(float* y) { y[0] = 1.f; }\n")
    h0 = lb.source_hash("probe_kernel")
    f.write_text("// a comment\n__global__ void k(float* y) {\n    y[0] = 1.f;  /* same */\n}\n")
    assert lb.source_hash("probe_kernel") == h0
    f.write_text("__global__ void k(float* y) { y[0] = 2.f; }\n")
    assert lb.source_hash("probe_kernel") != h0

