"""Every function the C header declares carries a comment above it (its
meaning, arguments, ownership and errors), alone or shared with the
declaration just before it."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DECL = re.compile(r"^(smat_status_t|const char|void|int64_t|int32_t|int|double|float)\b[^;]*\(")


def test_every_declaration_is_commented():
    for name in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not name.endswith(".h"):
            continue
        lines = open(os.path.join(ROOT, "include", name)).read().split("\n")
        bare = []
        for i, line in enumerate(lines):
            if not DECL.match(line):
                continue
            j = i - 1
            while j >= 0 and lines[j].strip() == "":
                j -= 1
            prev = lines[j].strip() if j >= 0 else ""
            # a comment right above, or a declaration it shares a comment with
            grouped = prev.endswith(");") and j > 0 and (i - j) == 1
            if not (prev.endswith("*/") or grouped):
                bare.append(f"{name}:{i + 1}: {line.strip()}")
        assert not bare, "\n".join(bare)
