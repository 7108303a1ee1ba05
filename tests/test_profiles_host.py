"""The ncu summaries under profiles/ name commands that run committed files
only: every `python bench.py ...` line parses with bench.py's own argument
parser (so each --config and flag exists), every pytest target exists, and
every ncu line carries --clock-control none."""
import glob
import os
import shlex

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _commands():
    for path in sorted(glob.glob(os.path.join(ROOT, 'profiles', '*.md'))):
        text = open(path).read().replace('\\\n', ' ')
        for line in text.splitlines():
            line = line.strip()
            if line.startswith(('python ', 'ncu ')):
                yield os.path.basename(path), line


def test_profile_commands_are_runnable():
    import bench
    cmds = list(_commands())
    assert len(cmds) >= 8
    for name, line in cmds:
        words = shlex.split(line)
        if words[0] == 'ncu':
            assert '--clock-control' in words and words[words.index('--clock-control') + 1] == 'none', (name, line)
            words = words[words.index('python'):]
        if words[1] == 'bench.py':
            bench.make_parser().parse_args(words[2:])  # exits (SystemExit) on an unknown flag or config
        elif words[1:3] == ['-m', 'pytest']:
            target = words[3].split('::')[0]
            assert os.path.exists(os.path.join(ROOT, target)), (name, target)
        else:
            raise AssertionError((name, line))
