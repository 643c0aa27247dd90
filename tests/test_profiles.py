"""The ncu summaries under profiles/ must be reproducible from the repository: every script a quoted
command runs is a tracked file of the repository, and every summary names its command."""
import json
import os
import re
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _tracked():
    out = subprocess.run(["git", "ls-files"], cwd=ROOT, capture_output=True, text=True)
    if out.returncode != 0:
        return None
    return set(out.stdout.split())


def _summaries():
    d = os.path.join(ROOT, "profiles")
    return sorted(os.path.join(d, f) for f in os.listdir(d) if f.endswith((".md", ".txt", ".json")))


def test_profile_commands_run_committed_files_only():
    tracked = _tracked()
    for path in _summaries():
        text = open(path).read()
        if path.endswith(".json"):
            text = json.loads(text).get("command", "")
        scripts = re.findall(r"python3? (?:-m \S+ )?([\w./-]+\.py)", text)
        assert "ncu" in text or path.endswith(".json"), f"{path}: no ncu command quoted"
        assert scripts, f"{path}: no command that runs a repository script"
        for s in scripts:
            assert os.path.exists(os.path.join(ROOT, s)), f"{path}: {s} does not exist"
            assert not s.startswith("_work"), f"{path}: {s} is a working file"
            if tracked is not None:
                assert s in tracked, f"{path}: {s} is not tracked"
