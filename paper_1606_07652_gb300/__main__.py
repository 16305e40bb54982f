from paper_1606_07652_gb300.build import build

print(build(verbose=True))
