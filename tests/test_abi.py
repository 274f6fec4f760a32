"""The C-ABI library loads on a machine without a GPU and exports every entry
point that include/zk_b300.h declares; calls that need a device fail with an
error code instead of crashing."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            names |= set(re.findall(r"^(?:int|const char \*|unsigned long long)\s*(zk_\w+)\s*\(", src, re.M))
    return names


def test_library_exports_every_declared_symbol():
    import paper_2507_07031_b300 as z
    declared = _declared()
    assert len(declared) >= 15
    for name in declared:
        assert hasattr(z.lib, name), name
        assert name in z.EXPORTED, name


def test_error_paths_without_device():
    import paper_2507_07031_b300 as z
    assert z.zk_strerror(z.ZK_EINVAL).startswith("invalid")
    assert z.lib.zk_commit(None, None, 0, None, None) == z.ZK_EINVAL
    assert z.lib.zk_init(None, 0, 0) == z.ZK_EINVAL
    assert z.lib.zk_fold(None, None, None, None, None, None, None) == z.ZK_EINVAL
    assert z.lib.zk_field_op(7, z.ZK_FOP_MUL, None, None, None, 1, None) == z.ZK_EINVAL
    assert z.lib.zk_field_op(z.ZK_FIELD_Q, z.ZK_FOP_MUL, None, None, None, 1, None) == z.ZK_EINVAL
    assert z.lib.zk_field_op(z.ZK_FIELD_Q, z.ZK_FOP_MULC + 1, None, None, None, 1, None) == z.ZK_EINVAL
    assert z.lib.zk_field_op(z.ZK_FIELD_Q, z.ZK_FOP_MULSUB, None, None, None, 1, None) == z.ZK_EINVAL
